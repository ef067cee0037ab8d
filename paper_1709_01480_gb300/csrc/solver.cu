// First-kind mobility solve (Sec. 3.1, Eq. discreteSaddlePoint) by right-
// preconditioned flexible GMRES with the block-diagonal preconditioner of
// Sec. 3.4 (Eqs. preconditionerGMRES, approximate-body-mobility, M-block-inverse).
//
// Unknowns x = [mu; U] (2N + 3 n_b, FP64); the saddle operator is
//     A x = [ M mu - K U ; -K^T mu ],  right-hand side b = -[slip; F].
// The preconditioner solves, body by body, [[M~, -K], [-K^T, 0]] [mu; U] = [r_mu; r_U]
// with M~_bb^+ = R_b M_ref^+ R_b^T:
//     z = R^T r_mu,  g = M_ref^+ z  (one GEMM over all bodies),
//     U' = -N~_ref (R^T r_U + K_ref^T g),  mu' = g + H U'  (H = M_ref^+ K_ref),
//     mu = R mu',  U = R U'   (R acts on (u_x, u_y) and leaves omega alone),
// where N~_ref = (K_ref^T M_ref^+ K_ref)^-1 is 3 x 3.  M_ref is the reference
// body alone in the periodic box (host-built, eigendecomposed with cuSOLVER);
// eigenvalues below 1e-12 of the largest in magnitude are dropped from the
// pseudo-inverse (a slightly negative near-null mode is kept, not dropped).
//
// Precision: FBIM_FP64 handles run FGMRES on the FP64 operator.  FBIM_FP32
// handles run iterative refinement: the outer residual b - A x uses the FP64
// operator; each correction is an FGMRES solve with the FP32 operator and an
// FP32 preconditioner GEMM; Krylov vectors and orthogonalisation stay FP64.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "fbim_internal.h"

#include "solver.cuh"

namespace fbim {

namespace {

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_rot_in(int N, int n_p, const double* __restrict__ rot, const double* __restrict__ in,
                         T* __restrict__ z) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    int b = m / n_p;
    const double2 u = reinterpret_cast<const double2*>(in)[m];
    if constexpr (std::is_same<T, float>::value) {
        // an FP32 preconditioner rotates in FP32 (GB300's FP64 pipe is ~1/74 of its FP32 rate)
        const float c = (float)rot[2 * b], s = (float)rot[2 * b + 1], ux = (float)u.x, uy = (float)u.y;
        reinterpret_cast<float2*>(z)[m] = make_float2(fmaf(c, ux, s * uy), fmaf(-s, ux, c * uy));
    } else {
        const double c = rot[2 * b], s = rot[2 * b + 1];
        z[2 * m] = c * u.x + s * u.y;
        z[2 * m + 1] = -s * u.x + c * u.y;
    }
}

// One block per body: U' = -N~ (R^T r_U + K_ref^T g), mu = R (g + H U'), with K_ref^T g
// formed as H^T z (z = R^T r_mu, g = M_ref^+ z; M_ref^+ symmetric): g carries large
// components along the near-null normal modes that K_ref^T cancels, z and H do not.
template <typename T>
__global__ void k_body_solve(int n_p, const double* __restrict__ ref, const double* __restrict__ rot,
                             const T* __restrict__ z, const T* __restrict__ g, const T* __restrict__ H,
                             const double* __restrict__ rU, double nt0, double nt1, double nt2, double nt3,
                             double nt4, double nt5, double nt6, double nt7, double nt8, double* __restrict__ out_mu,
                             double* __restrict__ out_U) {
    const int b = blockIdx.x;
    const int n2 = 2 * n_p;
    const T* gb = g + (size_t)b * n2;
    const T* zb = z + (size_t)b * n2;
    // sums over the body's nodes in T (an FP32 preconditioner stays off the FP64 pipe),
    // the 3x3 solve in FP64
    T sx = 0, sy = 0, st = 0;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        const T zi = zb[i];
        sx += H[i] * zi;
        sy += H[n2 + i] * zi;
        st += H[2 * n2 + i] * zi;
    }
    (void)ref;
    __shared__ T red[3][32];
    __shared__ double Up[3];
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        st += __shfl_xor_sync(0xffffffffu, st, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        red[0][warp] = sx;
        red[1][warp] = sy;
        red[2][warp] = st;
    }
    __syncthreads();
    const double c = rot[2 * b], s = rot[2 * b + 1];
    if (threadIdx.x == 0) {
        double tx = 0, ty = 0, tt = 0;
        for (int w = 0; w < nw; ++w) {
            tx += red[0][w];
            ty += red[1][w];
            tt += red[2][w];
        }
        // R^T r_U + K_ref^T g
        double ax = c * rU[3 * b] + s * rU[3 * b + 1] + tx;
        double ay = -s * rU[3 * b] + c * rU[3 * b + 1] + ty;
        double at = rU[3 * b + 2] + tt;
        double u0 = -(nt0 * ax + nt1 * ay + nt2 * at);
        double u1 = -(nt3 * ax + nt4 * ay + nt5 * at);
        double u2 = -(nt6 * ax + nt7 * ay + nt8 * at);
        Up[0] = u0;
        Up[1] = u1;
        Up[2] = u2;
        out_U[3 * b] = c * u0 - s * u1;
        out_U[3 * b + 1] = s * u0 + c * u1;
        out_U[3 * b + 2] = u2;
    }
    __syncthreads();
    const T u0 = (T)Up[0], u1 = (T)Up[1], u2 = (T)Up[2], cT = (T)c, sT = (T)s;
    for (int i = threadIdx.x; i < n_p; i += blockDim.x) {
        const T mx = gb[2 * i] + H[2 * i] * u0 + H[n2 + 2 * i] * u1 + H[2 * n2 + 2 * i] * u2;
        const T my = gb[2 * i + 1] + H[2 * i + 1] * u0 + H[n2 + 2 * i + 1] * u1 + H[2 * n2 + 2 * i + 1] * u2;
        const size_t m = (size_t)b * n_p + i;
        reinterpret_cast<double2*>(out_mu)[m] = make_double2((double)(cT * mx - sT * my), (double)(sT * mx + cT * my));
    }
}

// y_mu -= K U at every node; y_U = -K^T mu per body (one block per body).  The
// arithmetic is in T: the FP32 operator's saddle coupling stays off the FP64 pipe.
template <typename T>
__global__ void k_saddle_K(int n_p, const double* __restrict__ ref, const double* __restrict__ rot,
                           const double* __restrict__ mu, const double* __restrict__ U, double* __restrict__ ymu,
                           double* __restrict__ yU) {
    const int b = blockIdx.x;
    const T c = (T)rot[2 * b], s = (T)rot[2 * b + 1];
    const T ux = (T)U[3 * b], uy = (T)U[3 * b + 1], om = (T)U[3 * b + 2];
    T fx = 0, fy = 0, tq = 0;
    for (int j = threadIdx.x; j < n_p; j += blockDim.x) {
        // x - q = R gamma_ref
        const T gx = (T)ref[2 * j], gy = (T)ref[2 * j + 1];
        const T rx = c * gx - s * gy, ry = s * gx + c * gy;
        const size_t m = (size_t)b * n_p + j;
        double2 y = reinterpret_cast<double2*>(ymu)[m];
        y.x -= (double)(ux - om * ry);
        y.y -= (double)(uy + om * rx);
        reinterpret_cast<double2*>(ymu)[m] = y;
        const double2 mv = reinterpret_cast<const double2*>(mu)[m];
        const T mx = (T)mv.x, my = (T)mv.y;
        fx += mx;
        fy += my;
        tq += rx * my - ry * mx;
    }
    __shared__ T red[3][32];
    for (int o = 16; o > 0; o >>= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
        tq += __shfl_xor_sync(0xffffffffu, tq, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        red[0][warp] = fx;
        red[1][warp] = fy;
        red[2][warp] = tq;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, bb = 0, cc = 0;
        for (int w = 0; w < nw; ++w) {
            a += red[0][w];
            bb += red[1][w];
            cc += red[2][w];
        }
        yU[3 * b] = -a;
        yU[3 * b + 1] = -bb;
        yU[3 * b + 2] = -cc;
    }
}

__global__ void k_axpby(int n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = a * x[i] + b * y[i];
}

__global__ void k_neg_rhs(int n_mu, int n_U, const double* __restrict__ slip, const double* __restrict__ F,
                          double* __restrict__ b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_mu)
        b[i] = slip ? -slip[i] : 0.0;
    else if (i < n_mu + n_U)
        b[i] = -F[i - n_mu];
}

// A deterministic vector of uniform values in [-1, 1) (a 32-bit integer hash of the
// index): the probe vector of the FP32 operator's error estimate.
__global__ void k_probe_vector(int n, double* __restrict__ v) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned x = (unsigned)i * 2654435761u + 0x9e3779b9u;
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    v[i] = (double)x * (2.0 / 4294967296.0) - 1.0;
}

__global__ void k_check_finite(int n, const double* __restrict__ x, int* __restrict__ flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !isfinite(x[i])) atomicOr(flag, 1);
}

// ---------------------------------------------------------------------------
// The Arnoldi step on the device.  *kd is the index k of the newest basis vector,
// the one the step expands, so that one captured graph serves every k.  Row k of
// the step history holds the step's Gram-Schmidt coefficients (first pass at 0,
// second at m+1), |w|^2 at 2(m+1) and 1/|w| at 2(m+1)+1; the last sweep also
// copies the row to mapped host memory, where the host reads it after the step's
// event.  Classical Gram-Schmidt, fused: dots of w with the K = k+1 basis vectors,
// then w -= V h with the next pass's dots (or |w|^2) in the same sweep.  Each
// block owns CG_CHUNK consecutive entries (strided per thread for coalescing) and
// writes one partial per dot; the sweep's last block to finish sums the partials
// in a fixed order, so the result does not depend on scheduling.
// ---------------------------------------------------------------------------
constexpr int CG_TB = 256, CG_EPT = 4, CG_CHUNK = CG_TB * CG_EPT, CG_KCH = 64;

__host__ __device__ inline int hist_stride(int m) { return 2 * (m + 1) + 2; }

__device__ __forceinline__ double warp_sum(double s) {
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// part[j * nb + b] = sum over block b's entries of V_j w (j < K), or of w w (K = 0 -> one
// slot); CG_KCH dots at a time through shared memory
__device__ __forceinline__ void cgs_block_dots(int n, int K, const double* __restrict__ V, int ld, const double* wv,
                                               int nb, double* __restrict__ part, double (*red)[8]) {
    const int b = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i0 = b * CG_CHUNK + threadIdx.x;
    const int KK = K > 0 ? K : 1;
    for (int j0 = 0; j0 < KK; j0 += CG_KCH) {
        const int j1 = min(KK, j0 + CG_KCH);
        for (int j = j0; j < j1; ++j) {
            double sacc = 0.0;
            if (K > 0) {
                const double* v = V + (size_t)j * ld;
#pragma unroll
                for (int e = 0; e < CG_EPT; ++e) {
                    const int i = i0 + e * CG_TB;
                    if (i < n) sacc = fma(v[i], wv[e], sacc);
                }
            } else {
#pragma unroll
                for (int e = 0; e < CG_EPT; ++e) sacc = fma(wv[e], wv[e], sacc);
            }
            sacc = warp_sum(sacc);
            if (lane == 0) red[j - j0][warp] = sacc;
        }
        __syncthreads();
        for (int j = j0 + threadIdx.x; j < j1; j += CG_TB) {
            double t = 0.0;
            for (int q = 0; q < CG_TB / 32; ++q) t += red[j - j0][q];
            part[(size_t)j * nb + b] = t;
        }
        __syncthreads();
    }
}

// After every block has written its partials: the last block to arrive (an atomic
// count, which that block resets) returns true, behind a fence that makes the other
// blocks' partials visible to it.
__device__ __forceinline__ bool cgs_last_block(unsigned* __restrict__ count) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(count, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// out[j] = sum_b part[j nb + b] for j < K: a warp per j, its lanes strided over the
// blocks, then a warp sum (a fixed order)
__device__ __forceinline__ void cgs_sum_partials(int K, int nb, const double* part, double* __restrict__ out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = warp; j < K; j += nw) {
        double s = 0.0;
        for (int b = lane; b < nb; b += 32) s += __ldcg(part + (size_t)j * nb + b);
        s = warp_sum(s);
        if (lane == 0) out[j] = s;
    }
}

// first pass: partial dots of w with V_0..V_k; also stores the step's preconditioned
// vector z as Z_k (Z non-null)
__global__ void __launch_bounds__(CG_TB) k_cgs_dots(int n, const int* __restrict__ kd, const double* __restrict__ V,
                                                    int ld, const double* __restrict__ w, const double* __restrict__ z,
                                                    double* __restrict__ Z, int nb, double* __restrict__ part,
                                                    double* __restrict__ hist, int m, unsigned* __restrict__ count) {
    __shared__ double red[CG_KCH][8];
    const int k = *kd;
    double wv[CG_EPT];
    const int i0 = blockIdx.x * CG_CHUNK + threadIdx.x;
#pragma unroll
    for (int e = 0; e < CG_EPT; ++e) {
        const int i = i0 + e * CG_TB;
        wv[e] = i < n ? w[i] : 0.0;
    }
    cgs_block_dots(n, k + 1, V, ld, wv, nb, part, red);
    if (Z) {  // (the Lanczos iteration keeps no preconditioned basis)
#pragma unroll
        for (int e = 0; e < CG_EPT; ++e) {
            const int i = i0 + e * CG_TB;
            if (i < n) Z[(size_t)k * ld + i] = z[i];
        }
    }
    if (cgs_last_block(count)) {  // the first pass's coefficients into history row k
        cgs_sum_partials(k + 1, nb, part, hist + (size_t)k * hist_stride(m));
        if (threadIdx.x == 0) *count = 0u;
    }
}

// w -= sum_{j<=k} V_j h_j with h the history row's pass at offset off, then the partial
// dots of the new w with V (dots = 1) or |w|^2 (dots = 0).  The last block sums them:
// the second pass's coefficients into the row at m+1, or |w|^2 and 1/|w| (0 when w = 0)
// at 2(m+1) and 2(m+1)+1, the row to the host mirror and k + 1 into *kd.
__global__ void __launch_bounds__(CG_TB) k_cgs_update(int n, int* __restrict__ kd, const double* __restrict__ V,
                                                      int ld, double* __restrict__ hist, int m, int off,
                                                      double* __restrict__ w, int dots, int nb,
                                                      double* __restrict__ part, double* __restrict__ hist_host,
                                                      unsigned* __restrict__ count) {
    __shared__ double red[CG_KCH][8];
    const int k = *kd, K = k + 1;
    const double* hrow = hist + (size_t)k * hist_stride(m) + off;
    double wv[CG_EPT];
    const int i0 = blockIdx.x * CG_CHUNK + threadIdx.x;
#pragma unroll
    for (int e = 0; e < CG_EPT; ++e) {
        const int i = i0 + e * CG_TB;
        wv[e] = i < n ? w[i] : 0.0;
    }
    for (int j = 0; j < K; ++j) {
        const double* v = V + (size_t)j * ld;
        const double hj = hrow[j];
#pragma unroll
        for (int e = 0; e < CG_EPT; ++e) {
            const int i = i0 + e * CG_TB;
            if (i < n) wv[e] = fma(-v[i], hj, wv[e]);
        }
    }
#pragma unroll
    for (int e = 0; e < CG_EPT; ++e) {
        const int i = i0 + e * CG_TB;
        if (i < n) w[i] = wv[e];
    }
    cgs_block_dots(n, dots ? K : 0, V, ld, wv, nb, part, red);
    if (!cgs_last_block(count)) return;
    const int hs = hist_stride(m);
    double* row = hist + (size_t)k * hs;
    if (dots) {
        cgs_sum_partials(K, nb, part, row + (m + 1));
    } else {
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            double sq = 0.0;
            for (int b = lane; b < nb; b += 32) sq += __ldcg(part + b);
            sq = warp_sum(sq);
            if (lane == 0) {
                row[2 * (m + 1)] = sq;
                row[2 * (m + 1) + 1] = sq > 0.0 ? 1.0 / sqrt(sq) : 0.0;
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < hs; i += blockDim.x) hist_host[(size_t)k * hs + i] = row[i];
        __syncthreads();
        if (threadIdx.x == 0) *kd = k + 1;
    }
    if (threadIdx.x == 0) *count = 0u;
}

// V_{k+1} = w / |w| (k + 1 = *kd after the last update), also into the step input y2
__global__ void k_normalize(int n, const int* __restrict__ kd, const double* __restrict__ hist, int m,
                            const double* __restrict__ w, double* __restrict__ V, int ld, double* __restrict__ y2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k1 = *kd;
    const double a = hist[(size_t)(k1 - 1) * hist_stride(m) + 2 * (m + 1) + 1];
    const double v = a * w[i];
    V[(size_t)k1 * ld + i] = v;
    y2[i] = v;
}

// V_0 = a w, also into the step input y2; *kd = 0
__global__ void k_start(int n, double a, const double* __restrict__ w, double* __restrict__ V,
                        double* __restrict__ y2, int* __restrict__ kd) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *kd = 0;
    if (i >= n) return;
    const double v = a * w[i];
    V[i] = v;
    y2[i] = v;
}

// <x, y> over n entries: per-block partials, the last block to finish sums them in a
// fixed order (the result does not depend on scheduling) into *out (mapped host memory)
__global__ void __launch_bounds__(CG_TB) k_dot(int n, const double* __restrict__ x, const double* __restrict__ y,
                                               double* __restrict__ part, unsigned* __restrict__ count,
                                               double* __restrict__ out) {
    __shared__ double red[CG_TB / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double sacc = 0.0;
#pragma unroll
    for (int e = 0; e < CG_EPT; ++e) {
        const int i = blockIdx.x * CG_CHUNK + threadIdx.x + e * CG_TB;
        if (i < n) sacc = fma(x[i], y[i], sacc);
    }
    sacc = warp_sum(sacc);
    if (lane == 0) red[warp] = sacc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < CG_TB / 32; ++q) t += red[q];
        part[blockIdx.x] = t;
    }
    if (!cgs_last_block(count)) return;
    if (threadIdx.x < 32) {
        double t = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(part + b);
        t = warp_sum(t);
        if (lane == 0) {
            *out = t;
            *count = 0u;
        }
    }
}

// y = beta y + sum_{j < k} c_j V_j (a basis combination; c on the device)
__global__ void k_combine_basis(int n, int k, const double* __restrict__ V, int ld, const double* __restrict__ c,
                                double beta, double* __restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = beta == 0.0 ? 0.0 : beta * y[i];
    for (int j = 0; j < k; ++j) acc = fma(c[j], V[(size_t)j * ld + i], acc);
    y[i] = acc;
}

}  // namespace

// <x, y> for vectors of n <= the solver's length, on the handle's stream (host-synchronising)
fbim_status dev_dot(fbim_handle_s* h, int n, const double* x, const double* y, double& out) {
    Solver* S = h->solver;
    const int nb = (n + CG_CHUNK - 1) / CG_CHUNK;
    k_dot<<<nb, CG_TB, 0, h->stream>>>(n, x, y, S->dot_part, S->dot_count, S->dot_map);
    h->launches += 1;
    FBIM_CUDA_TRY(h, cudaGetLastError());
    FBIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    out = *(volatile double*)S->dot_host;
    return FBIM_OK;
}

fbim_status dev_norm2(fbim_handle_s* h, int n, const double* x, double& out) {
    double d = 0.0;
    FBIM_TRY(dev_dot(h, n, x, x, d));
    out = std::sqrt(std::max(d, 0.0));
    return FBIM_OK;
}

void dev_combine(fbim_handle_s* h, int n, int k, const double* V, int ld, const double* c, double beta, double* y) {
    k_combine_basis<<<(n + 255) / 256, 256, 0, h->stream>>>(n, k, V, ld, c, beta, y);
    h->launches += 1;
}

// Device-driven classical Gram-Schmidt on a basis of rows V_j (stride ld): see k_cgs_dots.
fbim_status cgs_alloc(fbim_handle_s* h, CgsState& c, int n, int ld, int m) {
    cgs_free(c);
    c.n = n;
    c.ld = ld;
    c.m = m;
    c.nb = (n + CG_CHUNK - 1) / CG_CHUNK;
    const size_t hist_bytes = sizeof(double) * (m + 1) * hist_stride(m);
    FBIM_CUDA_TRY(h, cudaMalloc(&c.kd, sizeof(int)));
    FBIM_CUDA_TRY(h, cudaMalloc(&c.count, sizeof(unsigned)));
    FBIM_CUDA_TRY(h, cudaMemsetAsync(c.count, 0, sizeof(unsigned), h->stream));
    FBIM_CUDA_TRY(h, cudaMalloc(&c.hist, hist_bytes));
    FBIM_CUDA_TRY(h, cudaMemsetAsync(c.hist, 0, hist_bytes, h->stream));
    FBIM_CUDA_TRY(h, cudaMalloc(&c.part, sizeof(double) * (m + 1) * c.nb));
    FBIM_CUDA_TRY(h, cudaHostAlloc(&c.hist_host, hist_bytes, cudaHostAllocMapped));
    memset(c.hist_host, 0, hist_bytes);
    FBIM_CUDA_TRY(h, cudaHostGetDevicePointer(&c.hist_map, c.hist_host, 0));
    return FBIM_OK;
}

void cgs_free(CgsState& c) {
    cudaFree(c.kd);
    cudaFree(c.count);
    cudaFree(c.hist);
    cudaFree(c.part);
    if (c.hist_host) cudaFreeHost(c.hist_host);
    c = CgsState();
}

int cgs_hist_stride(int m) { return hist_stride(m); }

// V_0 = a w (also into next_in), step index 0
void cgs_start(fbim_handle_s* h, CgsState& c, double a, const double* w, double* V, double* next_in) {
    k_start<<<(c.n + 255) / 256, 256, 0, h->stream>>>(c.n, a, w, V, next_in, c.kd);
    h->launches += 1;
}

// Orthonormalise w against V_0..V_k (k = the device's step index) by classical Gram-Schmidt
// (two passes or one), record the coefficients, |w|^2 and 1/|w| in history row k (and its
// mapped host copy), then V_{k+1} = w / |w|, also into next_in; the step index advances.
void cgs_step(fbim_handle_s* h, CgsState& c, double* V, double* w, bool two_pass, double* next_in) {
    const cudaStream_t st = h->stream;
    k_cgs_dots<<<c.nb, CG_TB, 0, st>>>(c.n, c.kd, V, c.ld, w, nullptr, nullptr, c.nb, c.part, c.hist, c.m, c.count);
    if (two_pass) {
        k_cgs_update<<<c.nb, CG_TB, 0, st>>>(c.n, c.kd, V, c.ld, c.hist, c.m, 0, w, 1, c.nb, c.part, c.hist_map,
                                             c.count);
        k_cgs_update<<<c.nb, CG_TB, 0, st>>>(c.n, c.kd, V, c.ld, c.hist, c.m, c.m + 1, w, 0, c.nb, c.part,
                                             c.hist_map, c.count);
    } else {
        k_cgs_update<<<c.nb, CG_TB, 0, st>>>(c.n, c.kd, V, c.ld, c.hist, c.m, 0, w, 0, c.nb, c.part, c.hist_map,
                                             c.count);
    }
    k_normalize<<<(c.n + 255) / 256, 256, 0, st>>>(c.n, c.kd, c.hist, c.m, w, V, c.ld, next_in);
    h->launches += two_pass ? 4 : 3;
}

namespace {

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
#define FBIM_CUBLAS_TRY(h, expr)                                                        \
    do {                                                                                \
        cublasStatus_t s__ = (expr);                                                    \
        if (s__ != CUBLAS_STATUS_SUCCESS) {                                             \
            (h)->fail(std::string(#expr) + ": cublas error " + std::to_string((int)s__)); \
            return FBIM_ERR_CUDA;                                                       \
        }                                                                               \
    } while (0)

// Symmetric eigendecomposition of A (row-major n x n, symmetric) with cuSOLVER.
fbim_status eig_sym(fbim_handle_s* h, const std::vector<double>& A, int n, std::vector<double>& lam,
                    std::vector<double>& V) {
    cusolverDnHandle_t sol = nullptr;
    if (cusolverDnCreate(&sol) != CUSOLVER_STATUS_SUCCESS) {
        h->fail("cusolverDnCreate failed");
        return FBIM_ERR_CUDA;
    }
    cusolverDnSetStream(sol, h->stream);
    double *dA = nullptr, *dW = nullptr, *work = nullptr;
    int* info = nullptr;
    int lwork = 0;
    fbim_status st = FBIM_OK;
    auto done = [&]() {
        cudaFree(dA);
        cudaFree(dW);
        cudaFree(work);
        cudaFree(info);
        cusolverDnDestroy(sol);
    };
    if (cudaMalloc(&dA, sizeof(double) * n * n) != cudaSuccess || cudaMalloc(&dW, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc(&info, sizeof(int)) != cudaSuccess) {
        done();
        h->fail("eig_sym: allocation failed");
        return FBIM_ERR_OOM;
    }
    cudaMemcpyAsync(dA, A.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice, h->stream);
    if (cusolverDnDsyevd_bufferSize(sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, dA, n, dW, &lwork) !=
            CUSOLVER_STATUS_SUCCESS ||
        cudaMalloc(&work, sizeof(double) * lwork) != cudaSuccess) {
        done();
        h->fail("eig_sym: workspace failed");
        return FBIM_ERR_CUDA;
    }
    if (cusolverDnDsyevd(sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, dA, n, dW, work, lwork, info) !=
        CUSOLVER_STATUS_SUCCESS) {
        done();
        h->fail("cusolverDnDsyevd failed");
        return FBIM_ERR_CUDA;
    }
    lam.resize(n);
    V.resize((size_t)n * n);
    int hinfo = 0;
    cudaMemcpyAsync(lam.data(), dW, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream);
    cudaMemcpyAsync(V.data(), dA, sizeof(double) * n * n, cudaMemcpyDeviceToHost, h->stream);
    cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess || hinfo != 0) {
        h->fail("eig_sym: eigensolver did not converge");
        st = FBIM_ERR_SETUP;
    }
    done();
    // V is column-major from cuSOLVER (symmetric input): column k = eigenvector k
    return st;
}

template <typename Dst>
fbim_status upload(fbim_handle_s* h, Dst** dst, const std::vector<double>& src) {
    std::vector<Dst> tmp(src.begin(), src.end());
    FBIM_CUDA_TRY(h, cudaMalloc(dst, sizeof(Dst) * tmp.size()));
    FBIM_CUDA_TRY(h, cudaMemcpyAsync(*dst, tmp.data(), sizeof(Dst) * tmp.size(), cudaMemcpyHostToDevice, h->stream));
    FBIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return FBIM_OK;
}

// f(A) = V diag(f(lam)) V^T over the eigenvalues kept (others -> 0); row-major result.
// signed = true keeps |lam| > rel max|lam| (pseudo-inverse of an indefinite block);
// signed = false keeps lam > rel max|lam| (square roots: non-positive modes are spurious).
std::vector<double> matrix_function(const std::vector<double>& lam, const std::vector<double>& V, int n, double rel,
                                    double (*f)(double), bool keep_negative) {
    double lmax = 0;
    for (double l : lam) lmax = std::max(lmax, std::fabs(l));
    std::vector<double> fl(n, 0.0);
    for (int k = 0; k < n; ++k)
        if ((keep_negative ? std::fabs(lam[k]) : lam[k]) > rel * lmax) fl[k] = f(lam[k]);
    std::vector<double> out((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double acc = 0;
            for (int k = 0; k < n; ++k) acc += V[(size_t)k * n + i] * fl[k] * V[(size_t)k * n + j];
            out[(size_t)i * n + j] = acc;
        }
    return out;
}

fbim_status setup_solver(fbim_handle_s* h) {
    if (h->solver) return FBIM_OK;
    Solver* S = new Solver();
    h->solver = S;
    const int n_p = h->n_p, n2 = 2 * n_p;
    S->n2 = n2;
    S->n = 2 * h->N + 3 * h->n_b;
    S->ld = (S->n + 31) / 32 * 32;
    S->restart = h->restart;
    std::vector<double> Mr, Mf;
    reference_blocks(h, h->host_band, Mr, Mf);
    // block preconditioner: M_ref^+, H = M_ref^+ K_ref, N~ = (K_ref^T M_ref^+ K_ref)^-1
    std::vector<double> lam, V;
    FBIM_TRY(eig_sym(h, Mf, n2, lam, V));
    // the Alpert correction can leave the near-null normal mode slightly negative:
    // the pseudo-inverse keeps it (it is a genuine eigenvalue of the block)
    std::vector<double> Mp = matrix_function(lam, V, n2, 1e-12, [](double l) { return 1.0 / l; }, true);
    const double* g = h->host_ref.data();
    std::vector<double> K((size_t)n2 * 3, 0.0);  // row-major n2 x 3
    for (int j = 0; j < n_p; ++j) {
        K[(2 * j) * 3 + 0] = 1.0;
        K[(2 * j + 1) * 3 + 1] = 1.0;
        K[(2 * j) * 3 + 2] = -g[2 * j + 1];
        K[(2 * j + 1) * 3 + 2] = g[2 * j];
    }
    std::vector<double> Hm((size_t)n2 * 3, 0.0);  // column-major n2 x 3
    for (int i = 0; i < n2; ++i)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int k = 0; k < n2; ++k) acc += Mp[(size_t)i * n2 + k] * K[k * 3 + c];
            Hm[(size_t)c * n2 + i] = acc;
        }
    double KH[9];
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int k = 0; k < n2; ++k) acc += K[k * 3 + a] * Hm[(size_t)c * n2 + k];
            KH[a * 3 + c] = acc;
        }
    // 3 x 3 inverse by cofactors
    double det = KH[0] * (KH[4] * KH[8] - KH[5] * KH[7]) - KH[1] * (KH[3] * KH[8] - KH[5] * KH[6]) +
                 KH[2] * (KH[3] * KH[7] - KH[4] * KH[6]);
    if (!(std::fabs(det) > 0)) {
        h->fail("reference body mobility is singular");
        return FBIM_ERR_SETUP;
    }
    double* N = S->Nt;
    N[0] = (KH[4] * KH[8] - KH[5] * KH[7]) / det;
    N[1] = (KH[2] * KH[7] - KH[1] * KH[8]) / det;
    N[2] = (KH[1] * KH[5] - KH[2] * KH[4]) / det;
    N[3] = (KH[5] * KH[6] - KH[3] * KH[8]) / det;
    N[4] = (KH[0] * KH[8] - KH[2] * KH[6]) / det;
    N[5] = (KH[2] * KH[3] - KH[0] * KH[5]) / det;
    N[6] = (KH[3] * KH[7] - KH[4] * KH[6]) / det;
    N[7] = (KH[1] * KH[6] - KH[0] * KH[7]) / det;
    N[8] = (KH[0] * KH[4] - KH[1] * KH[3]) / det;
    if (h->tensor_cores && h->precision == FBIM_FP32) {
        FBIM_CUDA_TRY(h, cudaMalloc(&S->tc_err, sizeof(int)));
        FBIM_CUDA_TRY(h, cudaMemsetAsync(S->tc_err, 0, sizeof(int), h->stream));
        FBIM_TRY(tc_prepare(h, Mp, n2, S->tc_Mp));
    }
    FBIM_TRY(upload(h, &S->Mpinv64, Mp));
    FBIM_TRY(upload(h, &S->Mpinv32, Mp));
    FBIM_TRY(upload(h, &S->H64, Hm));
    FBIM_TRY(upload(h, &S->H32, Hm));
    // Lanczos preconditioner: G_ref = M(r)_ref^{-1/2}, G_ref^+ = M(r)_ref^{1/2} (symmetric choice)
    std::vector<double> lr, Vr;
    FBIM_TRY(eig_sym(h, Mr, n2, lr, Vr));
    std::vector<double> G = matrix_function(lr, Vr, n2, 1e-12, [](double l) { return 1.0 / std::sqrt(l); }, false);
    std::vector<double> Gd = matrix_function(lr, Vr, n2, 1e-12, [](double l) { return std::sqrt(l); }, false);
    if (S->tc_err) {
        FBIM_TRY(tc_prepare(h, G, n2, S->tc_G));
        FBIM_TRY(tc_prepare(h, Gd, n2, S->tc_Gd));
    }
    FBIM_TRY(upload(h, &S->G64, G));
    FBIM_TRY(upload(h, &S->Gd64, Gd));
    FBIM_TRY(upload(h, &S->G32, G));
    FBIM_TRY(upload(h, &S->Gd32, Gd));
    // Krylov workspace
    const size_t n = S->n, m = S->restart, ld = S->ld;
    FBIM_CUDA_TRY(h, cudaMalloc(&S->V, sizeof(double) * ld * (m + 1)));
    FBIM_CUDA_TRY(h, cudaMalloc(&S->Z, sizeof(double) * ld * m));
    FBIM_CUDA_TRY(h, cudaMalloc(&S->w, sizeof(double) * n));
    FBIM_CUDA_TRY(h, cudaMalloc(&S->r, sizeof(double) * n));
    FBIM_CUDA_TRY(h, cudaMalloc(&S->d, sizeof(double) * n));
    FBIM_CUDA_TRY(h, cudaMalloc(&S->t, sizeof(double) * n));
    FBIM_CUDA_TRY(h, cudaMalloc(&S->corr, sizeof(double) * n));
    FBIM_CUDA_TRY(h, cudaMalloc(&S->hcol, sizeof(double) * (m + 1)));
    FBIM_CUDA_TRY(h, cudaMalloc(&S->gin, sizeof(double) * n));
    FBIM_CUDA_TRY(h, cudaMalloc(&S->cg_part, sizeof(double) * (m + 1) * ((n + CG_CHUNK - 1) / CG_CHUNK)));
    // device history; the host mirror has room for y after its rows
    const size_t hist_bytes = sizeof(double) * (m + 1) * hist_stride((int)m);
    FBIM_CUDA_TRY(h, cudaMalloc(&S->kd, sizeof(int)));
    FBIM_CUDA_TRY(h, cudaMemsetAsync(S->kd, 0, sizeof(int), h->stream));
    FBIM_CUDA_TRY(h, cudaMalloc(&S->cg_count, sizeof(unsigned)));
    FBIM_CUDA_TRY(h, cudaMemsetAsync(S->cg_count, 0, sizeof(unsigned), h->stream));
    FBIM_CUDA_TRY(h, cudaMalloc(&S->hist, hist_bytes));
    FBIM_CUDA_TRY(h, cudaMemsetAsync(S->hist, 0, hist_bytes, h->stream));
    FBIM_CUDA_TRY(h, cudaHostAlloc(&S->hist_host, hist_bytes + sizeof(double) * (m + 1), cudaHostAllocMapped));
    memset(S->hist_host, 0, hist_bytes + sizeof(double) * (m + 1));
    FBIM_CUDA_TRY(h, cudaHostGetDevicePointer(&S->hist_map, S->hist_host, 0));
    for (cudaEvent_t& ev : S->ev_step) FBIM_CUDA_TRY(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    FBIM_CUDA_TRY(h, cudaMalloc(&S->dot_part, sizeof(double) * ((n + CG_CHUNK - 1) / CG_CHUNK)));
    FBIM_CUDA_TRY(h, cudaMalloc(&S->dot_count, sizeof(unsigned)));
    FBIM_CUDA_TRY(h, cudaMemsetAsync(S->dot_count, 0, sizeof(unsigned), h->stream));
    FBIM_CUDA_TRY(h, cudaHostAlloc(&S->dot_host, sizeof(double), cudaHostAllocMapped));
    FBIM_CUDA_TRY(h, cudaHostGetDevicePointer(&S->dot_map, S->dot_host, 0));
    FBIM_CUDA_TRY(h, cudaMalloc(&S->gz, sizeof(double) * n));
    FBIM_CUDA_TRY(h, cudaMalloc(&S->gw, sizeof(double) * n));
    FBIM_CUDA_TRY(h, cudaMemsetAsync(S->gin, 0, sizeof(double) * n, h->stream));
    FBIM_CUDA_TRY(h, cudaMalloc(&S->zbuf, sizeof(double) * 2 * h->N));
    FBIM_CUDA_TRY(h, cudaMalloc(&S->gbuf, sizeof(double) * 2 * h->N));
    if (cublasCreate(&S->blas) != CUBLAS_STATUS_SUCCESS) {
        h->fail("cublasCreate failed");
        return FBIM_ERR_CUDA;
    }
    cublasSetStream(S->blas, h->stream);
    const size_t ws = 4u << 20;
    FBIM_CUDA_TRY(h, cudaMalloc(&S->blas_ws, ws));
    if (cublasSetWorkspace(S->blas, S->blas_ws, ws) != CUBLAS_STATUS_SUCCESS) {
        h->fail("cublasSetWorkspace failed");
        return FBIM_ERR_CUDA;
    }
    return FBIM_OK;
}

}  // namespace

void free_solver(fbim_handle_s* h) {
    Solver* S = h->solver;
    if (!S) return;
    for (void* p : {(void*)S->Mpinv64, (void*)S->Mpinv32, (void*)S->H64, (void*)S->H32, (void*)S->G64,
                    (void*)S->Gd64, (void*)S->G32, (void*)S->Gd32, (void*)S->V, (void*)S->Z, (void*)S->w,
                    (void*)S->r, (void*)S->d, (void*)S->t, (void*)S->hcol, S->zbuf, S->gbuf, (void*)S->lz,
                    (void*)S->lh, (void*)S->rfd, S->blas_ws, (void*)S->corr, (void*)S->gin, (void*)S->gz,
                    (void*)S->gw, (void*)S->cg_part, (void*)S->kd, (void*)S->hist, (void*)S->cg_count})
        cudaFree(p);
    if (S->hist_host) cudaFreeHost(S->hist_host);
    if (S->dot_host) cudaFreeHost(S->dot_host);
    cudaFree(S->dot_part);
    cudaFree(S->dot_count);
    cgs_free(S->lan);
    cudaFree(S->lan_in);
    cudaFree(S->lan_w);
    cudaFree(S->lan_c);
    tc_free(S->tc_Mp);
    tc_free(S->tc_G);
    tc_free(S->tc_Gd);
    cudaFree(S->tc_err);
    for (cudaEvent_t ev : S->ev_step)
        if (ev) cudaEventDestroy(ev);
    for (cudaGraphExec_t g : S->op_graph)
        if (g) cudaGraphExecDestroy(g);
    if (S->cap) cudaStreamDestroy(S->cap);
    if (S->blas) cublasDestroy(S->blas);
    delete S;
    h->solver = nullptr;
}

fbim_status ensure_solver(fbim_handle_s* h) { return setup_solver(h); }

// ---------------------------------------------------------------------------
// operators on x = [mu; U]
// ---------------------------------------------------------------------------
template <typename T>
static fbim_status saddle_apply(fbim_handle_s* h, const double* x, double* y) {
    const int N2 = 2 * h->N;
    FBIM_TRY(apply_operator<T>(h, x, y, 3));
    k_saddle_K<T><<<h->n_b, 128, 0, h->stream>>>(h->n_p, h->ref, h->rot, x, x + N2, y, y + N2);
    h->launches += 1;
    FBIM_CUDA_TRY(h, cudaGetLastError());
    return FBIM_OK;
}

template <typename T> struct Gemm;
template <> struct Gemm<double> {
    static cublasStatus_t run(cublasHandle_t b, int m, int n, int k, const double* A, const double* B, double* C) {
        const double one = 1.0, zero = 0.0;
        return cublasDgemm(b, CUBLAS_OP_N, CUBLAS_OP_N, m, n, k, &one, A, m, B, k, &zero, C, m);
    }
};
// The FP32 preconditioner's GEMM stays in full FP32: TF32 operands (10-bit mantissa)
// cost the FGMRES about 8% more iterations than they save in GEMM time.
template <> struct Gemm<float> {
    static cublasStatus_t run(cublasHandle_t b, int m, int n, int k, const float* A, const float* B, float* C) {
        const float one = 1.0f, zero = 0.0f;
        return cublasSgemm(b, CUBLAS_OP_N, CUBLAS_OP_N, m, n, k, &one, A, m, B, k, &zero, C, m);
    }
};

template <typename T>
static fbim_status precondition(fbim_handle_s* h, const double* in, double* out) {
    Solver* S = h->solver;
    const int N = h->N, N2 = 2 * N;
    T* z = (T*)S->zbuf;
    T* g = (T*)S->gbuf;
    if (std::is_same<T, float>::value && S->tc_Mp.ready) {
        // rotation, M_ref^+ contraction and body solve in one tensor-core kernel
        fbim_status cst = FBIM_OK;
        if (coarse_active(h, &cst)) {
            FBIM_TRY(tc_apply(h, S->tc_Mp, 1, in, nullptr, nullptr, (float*)g, nullptr, nullptr, S->tc_err));
            return coarse_body_solve<T>(h, g, (const T*)S->H32, in + N2, out, out + N2);
        }
        FBIM_TRY(cst);
        return tc_apply(h, S->tc_Mp, 2, in, out, out + N2, nullptr, S->H32, S->Nt, S->tc_err);
    }
    k_rot_in<T><<<(N + 255) / 256, 256, 0, h->stream>>>(N, h->n_p, h->rot, in, z);
    const T* Mp = std::is_same<T, float>::value ? (const T*)S->Mpinv32 : (const T*)S->Mpinv64;
    const T* Hm = std::is_same<T, float>::value ? (const T*)S->H32 : (const T*)S->H64;
    FBIM_CUBLAS_TRY(h, Gemm<T>::run(S->blas, S->n2, h->n_b, S->n2, Mp, z, g));
    fbim_status cst = FBIM_OK;
    if (coarse_active(h, &cst)) {
        FBIM_TRY(coarse_body_solve<T>(h, g, Hm, in + N2, out, out + N2));
        h->launches += 1;  // k_rot_in
        FBIM_CUDA_TRY(h, cudaGetLastError());
        return FBIM_OK;
    }
    FBIM_TRY(cst);
    const double* Nt = S->Nt;
    k_body_solve<T><<<h->n_b, 128, 0, h->stream>>>(h->n_p, h->ref, h->rot, z, g, Hm, in + N2, Nt[0], Nt[1],
                                                   Nt[2], Nt[3], Nt[4], Nt[5], Nt[6], Nt[7], Nt[8], out, out + N2);
    h->launches += 2;
    FBIM_CUDA_TRY(h, cudaGetLastError());
    return FBIM_OK;
}

// One Arnoldi step on the device (see k_cgs_dots): z = P v_k into gz and Z_k,
// w = A z into gw, orthogonalised against V_0..V_k (classical Gram-Schmidt: twice
// for FP64 solves; once for the FP32-operator corrections of refinement, which
// stop at ~1e-4, where the basis's loss of orthogonality, far below that, does not
// matter, the FP64 outer residual deciding the accuracy), then V_{k+1} = w / |w|,
// also into gin, the next step's input.
template <typename T>
static fbim_status arnoldi_step(fbim_handle_s* h) {
    Solver* S = h->solver;
    const int n = S->n, m = S->restart, ld = S->ld;
    const int nb = (n + CG_CHUNK - 1) / CG_CHUNK;
    const bool two_pass = !std::is_same<T, float>::value;
    FBIM_TRY(precondition<T>(h, S->gin, S->gz));
    FBIM_TRY(saddle_apply<T>(h, S->gz, S->gw));
    const cudaStream_t st = h->stream;
    k_cgs_dots<<<nb, CG_TB, 0, st>>>(n, S->kd, S->V, ld, S->gw, S->gz, S->Z, nb, S->cg_part, S->hist, m, S->cg_count);
    if (two_pass) {
        k_cgs_update<<<nb, CG_TB, 0, st>>>(n, S->kd, S->V, ld, S->hist, m, 0, S->gw, 1, nb, S->cg_part, S->hist_map,
                                           S->cg_count);
        k_cgs_update<<<nb, CG_TB, 0, st>>>(n, S->kd, S->V, ld, S->hist, m, m + 1, S->gw, 0, nb, S->cg_part,
                                           S->hist_map, S->cg_count);
    } else {
        k_cgs_update<<<nb, CG_TB, 0, st>>>(n, S->kd, S->V, ld, S->hist, m, 0, S->gw, 0, nb, S->cg_part, S->hist_map,
                                           S->cg_count);
    }
    k_normalize<<<(n + 255) / 256, 256, 0, st>>>(n, S->kd, S->hist, m, S->gw, S->V, ld, S->gin);
    h->launches += two_pass ? 4 : 3;
    FBIM_CUDA_TRY(h, cudaGetLastError());
    return FBIM_OK;
}

// The Arnoldi step captured once as a CUDA graph on fixed buffers, so that each
// step costs one graph launch instead of some thirty kernel, cuFFT and cuBLAS
// launches.  Recaptured when a buffer the launches hold by pointer was reallocated
// (layout_version).
template <typename T>
static fbim_status op_graph(fbim_handle_s* h) {
    Solver* S = h->solver;
    const int k = std::is_same<T, float>::value ? 0 : 1;
    if (S->op_graph[k] && S->op_version[k] == h->layout_version) return FBIM_OK;
    if (S->op_graph[k]) {
        cudaGraphExecDestroy(S->op_graph[k]);
        S->op_graph[k] = nullptr;
    }
    // warm-up outside the capture: first use allocates, plans and refreshes
    FBIM_TRY(precondition<T>(h, S->gin, S->gz));
    FBIM_TRY(saddle_apply<T>(h, S->gz, S->gw));
    FBIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (!S->cap) FBIM_CUDA_TRY(h, cudaStreamCreateWithFlags(&S->cap, cudaStreamNonBlocking));
    const cudaStream_t orig = h->stream;
    const bool timing = h->timing;
    const long long l0 = h->launches;
    h->timing = false;
    FBIM_CUDA_TRY(h, cudaStreamBeginCapture(S->cap, cudaStreamCaptureModeThreadLocal));
    bind_stream(h, S->cap);
    fbim_status st = arnoldi_step<T>(h);
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(S->cap, &graph);
    bind_stream(h, orig);
    h->timing = timing;
    S->op_kernels[k] = h->launches - l0;
    h->launches = l0;  // captured, not run
    if (st != FBIM_OK || ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (st != FBIM_OK) return st;
        h->fail(std::string("Arnoldi step capture: ") + cudaGetErrorString(ee));
        return FBIM_ERR_CUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&S->op_graph[k], graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        S->op_graph[k] = nullptr;
        h->fail(std::string("Arnoldi step graph instantiate: ") + cudaGetErrorString(ie));
        return FBIM_ERR_CUDA;
    }
    S->op_version[k] = h->layout_version;
    return FBIM_OK;
}

// Restarted flexible GMRES for A x = b with the operator and preconditioner in precision T.
// x holds the initial guess on entry.  Returns the iteration count and the estimated
// relative residual |b - A x| / |b| of the last cycle.
//
// The host keeps the Hessenberg matrix and its Givens rotations and reads each
// step's coefficients from the mapped history row after the step's event.  Step
// k+1 is queued before step k is read, so that the device does not wait for the
// host between steps, except where step k is predicted to converge (the last ratio
// of residual estimates carried one step on lands within 3 tol): a step run past
// convergence costs far more than the wait it saves.  A step queued past the end
// only writes V_{k+2}, Z_{k+1} and history row k+1, which the update x += Z y does
// not read.
// bnorm_in > 0 is |b| when the caller knows it (each norm costs a host sync).
template <typename T>
static fbim_status fgmres(fbim_handle_s* h, const double* b, double* x, double tol, int max_iter, int& iters,
                          double& rel_est, bool x_is_zero = false, bool trust_estimate = false,
                          double bnorm_in = 0.0) {
    Solver* S = h->solver;
    const int n = S->n, m = S->restart, ld = S->ld, hs = hist_stride(m);
    double bnorm = bnorm_in;
    if (!(bnorm > 0.0)) FBIM_TRY(dev_norm2(h, n, b, bnorm));
    iters = 0;
    rel_est = 0;
    if (bnorm == 0) {
        FBIM_CUDA_TRY(h, cudaMemsetAsync(x, 0, sizeof(double) * n, h->stream));
        return FBIM_OK;
    }
    std::vector<double> Hh((size_t)(m + 1) * m), cs(m), sn(m), gvec(m + 1);
    const bool use_graph = !h->timing;
    const bool two_pass = !std::is_same<T, float>::value;
    const int gk = std::is_same<T, float>::value ? 0 : 1;
    if (use_graph) {
        FBIM_TRY(coarse_refresh(h));  // host-synchronising, and may reallocate: before the graph check
        FBIM_TRY(op_graph<T>(h));
    }
    auto enqueue = [&](int k) -> fbim_status {
        if (use_graph) {
            FBIM_CUDA_TRY(h, cudaGraphLaunch(S->op_graph[gk], h->stream));
            h->launches += S->op_kernels[gk];
        } else {
            FBIM_TRY(arnoldi_step<T>(h));
        }
        FBIM_CUDA_TRY(h, cudaEventRecord(S->ev_step[k & 1], h->stream));
        return FBIM_OK;
    };
    const int tb = 256, nb = (n + tb - 1) / tb;
    bool first = true, recapture = false;
    while (true) {
        if (recapture && use_graph) FBIM_TRY(op_graph<T>(h));
        recapture = false;
        // r = b - A x (just b when the initial guess is zero)
        double beta = 0;
        if (first && x_is_zero) {
            FBIM_CUDA_TRY(h, cudaMemcpyAsync(S->w, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
            beta = bnorm;
        } else {
            FBIM_TRY(saddle_apply<T>(h, x, S->w));
            k_axpby<<<nb, tb, 0, h->stream>>>(n, 1.0, b, -1.0, S->w);  // w = b - w
            h->launches += 1;
            FBIM_TRY(dev_norm2(h, n, S->w, beta));
        }
        first = false;
        rel_est = beta / bnorm;
        if (!std::isfinite(beta)) {
            h->fail("GMRES residual is not finite");
            return FBIM_ERR_NONFINITE;
        }
        if (rel_est <= tol || iters >= max_iter) return FBIM_OK;
        k_start<<<nb, tb, 0, h->stream>>>(n, 1.0 / beta, S->w, S->V, S->gin, S->kd);
        h->launches += 1;
        std::fill(gvec.begin(), gvec.end(), 0.0);
        gvec[0] = beta;
        int k_used = 0;
        double res1 = rel_est, res2 = 0.0;  // residual estimates after the last two steps
        const double res_start = rel_est;
        // stagnation guard of the learned coarse level: a cycle that has not cut the
        // residual tenfold in kGuardSteps steps ends here, and the solve goes on with the
        // block-diagonal preconditioner (the coarse level stays off for this geometry)
        constexpr int kGuardSteps = 20;
        bool stagnated = false;
        FBIM_TRY(enqueue(0));
        for (int k = 0; k < m; ++k) {
            bool ahead = k + 1 < m && iters + 1 < max_iter;
            if (ahead) {
                const double rho = res2 > 0.0 ? std::min(res1 / res2, 1.0) : 1.0;
                ahead = res1 * rho > 3.0 * tol;
            }
            if (ahead) FBIM_TRY(enqueue(k + 1));
            FBIM_CUDA_TRY(h, cudaEventSynchronize(S->ev_step[k & 1]));
            const double* row = S->hist_host + (size_t)k * hs;
            const double hn = std::sqrt(std::max(row[2 * (m + 1)], 0.0));
            double* col = &Hh[(size_t)k * (m + 1)];
            for (int i = 0; i <= k; ++i) col[i] = two_pass ? row[i] + row[(m + 1) + i] : row[i];
            col[k + 1] = hn;
            if (!std::isfinite(hn)) {
                h->fail("GMRES iterate is not finite");
                return FBIM_ERR_NONFINITE;
            }
            for (int i = 0; i < k; ++i) {
                double t0 = cs[i] * col[i] + sn[i] * col[i + 1];
                col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
                col[i] = t0;
            }
            double den = std::hypot(col[k], col[k + 1]);
            cs[k] = den > 0 ? col[k] / den : 1.0;
            sn[k] = den > 0 ? col[k + 1] / den : 0.0;
            col[k] = den;
            col[k + 1] = 0;
            gvec[k + 1] = -sn[k] * gvec[k];
            gvec[k] = cs[k] * gvec[k];
            ++iters;
            k_used = k + 1;
            res2 = res1;
            res1 = std::fabs(gvec[k + 1]) / bnorm;
            if (res1 <= tol || iters >= max_iter || hn == 0) break;
            if (k + 1 == kGuardSteps && res1 > 0.1 * res_start && h->coarse &&
                h->coarse_suspended_geom != h->geom_version) {
                stagnated = true;
                break;
            }
            if (!ahead && k + 1 < m) FBIM_TRY(enqueue(k + 1));
        }
        // y = R^-1 g (upper triangular), x += Z y; y is staged in pinned memory after the
        // history rows (the previous cycle's copy was complete at this cycle's first sync)
        double* y = S->hist_host + (size_t)(m + 1) * hs;
        for (int i = k_used - 1; i >= 0; --i) {
            double acc = gvec[i];
            for (int j = i + 1; j < k_used; ++j) acc -= Hh[(size_t)j * (m + 1) + i] * y[j];
            y[i] = acc / Hh[(size_t)i * (m + 1) + i];
        }
        FBIM_CUDA_TRY(h, cudaMemcpyAsync(S->hcol, y, sizeof(double) * k_used, cudaMemcpyHostToDevice, h->stream));
        dev_combine(h, n, k_used, S->Z, ld, S->hcol, 1.0, x);
        if (stagnated) {
            h->coarse_suspended_geom = h->geom_version;
            ++h->coarse_fallbacks;
            ++h->layout_version;  // the captured step holds the coarse level: recapture
            recapture = true;
            continue;             // a new cycle from the true residual of the updated x
        }
        // A correction of iterative refinement stops on the cycle's own estimate: the
        // outer loop measures the true FP64 residual anyway, and a restart started only
        // because the FP32 residual lands just above the inner tolerance costs a cycle.
        if (trust_estimate && k_used > 0) {
            rel_est = std::fabs(gvec[k_used]) / bnorm;
            if (rel_est <= tol || iters >= max_iter) return FBIM_OK;
        }
    }
}

// True residual r = b - A_64 x with the FP64 operator, rn = |r| and rel = rn / bn
// (bn = |b|).
static fbim_status true_residual(fbim_handle_s* h, const double* b, const double* x, double* r, double bn,
                                 double& rn, double& rel) {
    Solver* S = h->solver;
    const int n = S->n;
    FBIM_TRY(saddle_apply<double>(h, x, r));
    k_axpby<<<(n + 255) / 256, 256, 0, h->stream>>>(n, 1.0, b, -1.0, r);
    h->launches += 1;
    rn = 0;
    FBIM_TRY(dev_norm2(h, n, r, rn));
    rel = bn > 0 ? rn / bn : 0.0;
    return FBIM_OK;
}

// e32 = |(A_32 - A_64) v| / |v| for the probe vector v (FP32 handles; once per handle).
static fbim_status measure_e32(fbim_handle_s* h) {
    Solver* S = h->solver;
    if (S->e32 >= 0.0) return FBIM_OK;
    const int n = S->n;
    k_probe_vector<<<(n + 255) / 256, 256, 0, h->stream>>>(n, S->corr);
    h->launches += 2;
    FBIM_TRY(saddle_apply<float>(h, S->corr, S->w));
    FBIM_TRY(saddle_apply<double>(h, S->corr, S->r));
    k_axpby<<<(n + 255) / 256, 256, 0, h->stream>>>(n, 1.0, S->r, -1.0, S->w);  // w = A_64 v - A_32 v
    double en = 0.0, vn = 0.0;
    FBIM_TRY(dev_norm2(h, n, S->w, en));
    FBIM_TRY(dev_norm2(h, n, S->corr, vn));
    S->e32 = vn > 0.0 ? en / vn : 0.0;
    return FBIM_OK;
}

// warm: start from the solution [mu; U] of the previous solve on this handle (kept in
// the solver's workspace) instead of zero, e.g. for a nearby configuration.
fbim_status mobility_solve(fbim_handle_s* h, const double* F, const double* slip, double tol, int max_iter,
                           double* U, double* mu_out, int* iters_out, double* res_out, bool warm) {
    FBIM_TRY(setup_solver(h));
    Solver* S = h->solver;
    const int n = S->n, N2 = 2 * h->N;
    const int tb = 256, nb = (n + tb - 1) / tb;
    // b lives in S->t, x in S->d
    k_neg_rhs<<<nb, tb, 0, h->stream>>>(N2, 3 * h->n_b, slip, F, S->t);
    h->launches += 1;
    warm = warm && S->have_x;
    if (!warm) FBIM_CUDA_TRY(h, cudaMemsetAsync(S->d, 0, sizeof(double) * n, h->stream));
    int iters = 0;
    double rel = 1.0, bn = 0.0, rn = 0.0;  // |r| / |b|, |b|, |r|
    FBIM_TRY(dev_norm2(h, n, S->t, bn));
    if (h->precision == FBIM_FP64) {
        double est = 0;
        FBIM_TRY(fgmres<double>(h, S->t, S->d, tol, max_iter, iters, est, !warm, false, bn));
        FBIM_TRY(true_residual(h, S->t, S->d, S->r, bn, rn, rel));
    } else {
        // Iterative refinement: FP32-operator corrections, FP64 residuals.  r holds the
        // residual b - A x and rel = |r| / |b|.  After a correction d computed from a
        // residual that is not yet small (see recompute_above), x has changed a lot and r is
        // recomputed from scratch with the FP64 operator.  After a later correction,
        // |d| ~ rel |x|, so the inner GMRES's own residual estimate gives the new rel and
        // r - A_32 d the new residual to within ~3e-7 rel |b| (the FP32 operator's
        // error on d): one FP64 matvec per solve instead of one per correction.
        double* corr = S->corr;
        fbim_status st = FBIM_OK;
        FBIM_TRY(measure_e32(h));  // uses corr, w and r as scratch: before r is set
        if (warm) {
            FBIM_TRY(true_residual(h, S->t, S->d, S->r, bn, rn, rel));
        } else {
            cudaMemcpyAsync(S->r, S->t, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream);  // x = 0
            rn = bn;
            rel = bn > 0 ? 1.0 : 0.0;
        }
        // The residual advanced with the FP32 operator errs by ~1e-6 rel_prev |b| (FP32
        // operator error with margin); it stays below 0.05 tol |b| while rel_prev <= 5e4 tol.
        const double recompute_above = std::max(1e-3, 5e4 * tol);
        // A residual advanced by r - A_32 d differs from the true b - A_64 x by (A_64 - A_32) d,
        // at most about e32 |d| (the FP32 operator's measured error per unit vector, with a
        // margin of 3).  That is small relative to |b| unless x, and so d, carries large
        // components the operator nearly annihilates (the first-kind system's near-null
        // normal modes).  drift accumulates the bound over the corrections since the last
        // FP64 residual; an estimate within tol of convergence only counts once estimate +
        // drift <= tol, else the residual is measured.
        double drift = 0.0;
        for (int outer = 0; outer < 40 && rel > tol && iters < max_iter; ++outer) {
            // Each correction solves A d = r with the FP32 operator to a relative 1e-4
            // (or tighter when that already meets tol), within one restart cycle: the
            // FP32 operator cannot resolve residuals much below ~1e-5 of a right-hand
            // side like the random slip, and refinement gains its factor per step.
            const double inner = std::max(0.3 * tol / rel, 1e-4);
            cudaMemsetAsync(corr, 0, sizeof(double) * n, h->stream);
            int it = 0;
            double est = 0;
            st = fgmres<float>(h, S->r, corr, inner, std::min(max_iter - iters, S->restart), it, est, true, true,
                               rn);
            if (st != FBIM_OK) break;
            iters += it;
            k_axpby<<<nb, tb, 0, h->stream>>>(n, 1.0, corr, 1.0, S->d);
            h->launches += 1;
            if (rel > recompute_above) {
                st = true_residual(h, S->t, S->d, S->r, bn, rn, rel);
                if (st != FBIM_OK) break;
                drift = 0.0;
            } else {
                const double rel_prev = rel;
                rel = est * rel_prev;
                double dn = 0.0;
                FBIM_TRY(dev_norm2(h, n, corr, dn));
                drift += 3.0 * S->e32 * dn / (bn > 0 ? bn : 1.0);
                if (rel <= tol && rel + drift > tol) {
                    // the estimate cannot vouch for convergence: measure
                    st = true_residual(h, S->t, S->d, S->r, bn, rn, rel);
                    if (st != FBIM_OK) break;
                    drift = 0.0;
                    continue;
                }
                if (rel > tol && iters < max_iter) {
                    // another correction follows: r <- r - A_32 d
                    FBIM_TRY(saddle_apply<float>(h, corr, S->w));
                    k_axpby<<<nb, tb, 0, h->stream>>>(n, -1.0, S->w, 1.0, S->r);
                    h->launches += 1;
                    FBIM_TRY(dev_norm2(h, n, S->r, rn));
                    rel = bn > 0 ? rn / bn : 0.0;
                }
            }
        }
        FBIM_TRY(st);
    }
    S->have_x = std::isfinite(rel);
    if (h->audit) {
        // measure the true FP64 residual of the returned [mu; U] beside the reported one
        double rn_true = 0.0, rel_true = 0.0;
        FBIM_TRY(true_residual(h, S->t, S->d, S->r, bn, rn_true, rel_true));
        h->audit_reported.push_back(rel);
        h->audit_measured.push_back(rel_true);
        if ((int)h->audit_reported.size() > fbim_handle_s::kAuditKeep) {
            h->audit_reported.erase(h->audit_reported.begin());
            h->audit_measured.erase(h->audit_measured.begin());
        }
    }
    FBIM_CUDA_TRY(h, cudaMemcpyAsync(U, S->d + N2, sizeof(double) * 3 * h->n_b, cudaMemcpyDeviceToDevice,
                                     h->stream));
    if (mu_out)
        FBIM_CUDA_TRY(h, cudaMemcpyAsync(mu_out, S->d, sizeof(double) * N2, cudaMemcpyDeviceToDevice, h->stream));
    FBIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    FBIM_TRY(tc_check(h));
    if (iters_out) *iters_out = iters;
    if (res_out) *res_out = rel;
    if (!std::isfinite(rel)) {
        h->fail("mobility solve produced non-finite values");
        return FBIM_ERR_NONFINITE;
    }
    if (rel > tol) {
        h->fail("GMRES reached the iteration cap before the tolerance");
        return FBIM_ERR_NOT_CONVERGED;
    }
    return FBIM_OK;
}

fbim_status set_residual_audit(fbim_handle_s* h, int on) {
    h->audit = on != 0;
    h->audit_reported.clear();
    h->audit_measured.clear();
    return FBIM_OK;
}

// exposed for the batched solver (batch.cu)
fbim_status solver_precondition(fbim_handle_s* h, const double* in, double* out, bool fp32) {
    return fp32 ? precondition<float>(h, in, out) : precondition<double>(h, in, out);
}

fbim_status solver_saddle(fbim_handle_s* h, const double* x, double* y, bool fp32) {
    return fp32 ? saddle_apply<float>(h, x, y) : saddle_apply<double>(h, x, y);
}

void bind_stream(fbim_handle_s* h, cudaStream_t s) {
    h->stream = s;
    if (h->e64.ready) {
        cufftSetStream(h->e64.plan_f, s);
        cufftSetStream(h->e64.plan_i, s);
    }
    if (h->e32.ready) {
        cufftSetStream(h->e32.plan_f, s);
        cufftSetStream(h->e32.plan_i, s);
    }
    if (h->solver && h->solver->blas) cublasSetStream(h->solver->blas, s);
}

}  // namespace fbim

extern "C" fbim_status fbim_precondition(fbim_handle h, const double* in_dev, double* out_dev) {
    if (!h || !in_dev || !out_dev) return FBIM_ERR_INVALID_ARG;
    if ((((uintptr_t)in_dev) | ((uintptr_t)out_dev)) & 15) {
        h->fail("fbim_precondition: in and out must be 16-byte aligned");
        return FBIM_ERR_INVALID_ARG;
    }
    try {
        if (cudaSetDevice(h->device) != cudaSuccess) return FBIM_ERR_CUDA;
        FBIM_TRY(fbim::ensure_solver(h));
        FBIM_TRY(fbim::solver_precondition(h, in_dev, out_dev, h->precision == FBIM_FP32));
        FBIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        return fbim::tc_check(h);
    } catch (...) {
        h->fail("unexpected host exception in fbim_precondition");
        return FBIM_ERR_SETUP;
    }
}

extern "C" fbim_status fbim_set_residual_audit(fbim_handle h, int on) {
    if (!h) return FBIM_ERR_INVALID_ARG;
    return fbim::set_residual_audit(h, on);
}

extern "C" fbim_status fbim_residual_audit(fbim_handle h, int n, double* reported, double* measured, int* count) {
    if (!h || n < 0 || (n > 0 && (!reported || !measured))) return FBIM_ERR_INVALID_ARG;
    const int have = (int)h->audit_reported.size();
    const int k = std::min(n, have);
    for (int i = 0; i < k; ++i) {
        reported[i] = h->audit_reported[have - k + i];
        measured[i] = h->audit_measured[have - k + i];
    }
    if (count) *count = k;
    return FBIM_OK;
}

extern "C" fbim_status fbim_mobility_solve(fbim_handle h, const double* F_dev, const double* slip_dev, double tol,
                                           int max_iter, double* U_dev, double* mu_dev, int* iters,
                                           double* rel_residual) {
    if (!h || !F_dev || !U_dev || !(tol > 0) || max_iter <= 0) return FBIM_ERR_INVALID_ARG;
    try {
        if (cudaSetDevice(h->device) != cudaSuccess) return FBIM_ERR_CUDA;
        return fbim::mobility_solve(h, F_dev, slip_dev, tol, max_iter, U_dev, mu_dev, iters, rel_residual, false);
    } catch (...) {
        h->fail("unexpected host exception in fbim_mobility_solve");
        return FBIM_ERR_SETUP;
    }
}
