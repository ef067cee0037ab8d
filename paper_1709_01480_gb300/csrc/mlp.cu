// Pair-correction network of the learned coarse level: 6 -> 128 -> 128 -> 128 -> 36,
// tanh hidden layers, linear output, trained with the mean squared error and Adam
// (Kingma & Ba, ICLR 2015, Algorithm 1).  The paper's preconditioner is the
// block-diagonal one of Sec. 3.4; the network only feeds the optional coarse level.
//
// Every matrix product (forward, input gradient, weight gradient) runs on the
// tensor cores: operands are rounded to bfloat16 when a 64x64 output tile's
// operand slices are staged in shared memory, products accumulate in FP32
// (mma.sync m16n8k16 bf16), and the epilogue adds the bias and applies tanh or
// the tanh derivative.  Master weights, biases, activations, gradients and the
// Adam moments are FP32.
//
// Parameter vector (FP32, 38564 entries): for l = 1..4, W_l [n_l][n_{l-1}]
// row-major, then b_l [n_l]; widths (6, 128, 128, 128, 36).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "fbim_internal.h"

namespace {

constexpr int kLayers = 4;
constexpr int kWidth[kLayers + 1] = {6, 128, 128, 128, 36};

int param_offset_W(int l) {
    int o = 0;
    for (int i = 0; i < l; ++i) o += kWidth[i + 1] * kWidth[i] + kWidth[i + 1];
    return o;
}
int param_offset_b(int l) { return param_offset_W(l) + kWidth[l + 1] * kWidth[l]; }
constexpr int kParams = 6 * 128 + 128 + 2 * (128 * 128 + 128) + 36 * 128 + 36;

// ---------------------------------------------------------------------------
// C[M][N] = sum_k A(m, k) B(k, n) (+ bias[n]), then the epilogue:
//   EPI_LINEAR: C = v;  EPI_TANH: C = tanh(v);  EPI_DTANH: C = v (1 - aux[m][n]^2).
// A(m, k) = A[m sam + k sak], B(k, n) = B[k sbk + n sbn] (FP32, rounded to bf16 on
// staging).  Tile 64 x 64 x 32, 4 warps of 32 x 32 each (2 x 4 m16n8 fragments).
// ---------------------------------------------------------------------------
enum { EPI_LINEAR = 0, EPI_TANH = 1, EPI_DTANH = 2 };
constexpr int BM = 64, BN = 64, BK = 32, PAD = 8, LDS = BK + PAD;

__device__ __forceinline__ void mma_bf16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

template <int EPI>
__global__ void __launch_bounds__(128) k_gemm_bf16(int M, int N, int K, const float* __restrict__ A, long long sam,
                                                   long long sak, const float* __restrict__ B, long long sbk,
                                                   long long sbn, const float* __restrict__ bias,
                                                   const float* __restrict__ aux, float* __restrict__ C, int ldc) {
    __shared__ __align__(16) __nv_bfloat16 As[BM][LDS];  // [m][k]
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][LDS];  // [n][k]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int e = tid; e < BM * BK; e += 128) {
            const int r = e / BK, c = e % BK;
            const int gm = m0 + r, gk = k0 + c;
            const float va = (gm < M && gk < K) ? A[(long long)gm * sam + (long long)gk * sak] : 0.f;
            As[r][c] = __float2bfloat16_rn(va);
            const int gn = n0 + r;
            const float vb = (gn < N && gk < K) ? B[(long long)gk * sbk + (long long)gn * sbn] : 0.f;
            Bs[r][c] = __float2bfloat16_rn(vb);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            unsigned a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r0 = wm * 32 + i * 16;
                a[i][0] = *reinterpret_cast<const unsigned*>(&As[r0 + g][kk + 2 * t]);
                a[i][1] = *reinterpret_cast<const unsigned*>(&As[r0 + g + 8][kk + 2 * t]);
                a[i][2] = *reinterpret_cast<const unsigned*>(&As[r0 + g][kk + 8 + 2 * t]);
                a[i][3] = *reinterpret_cast<const unsigned*>(&As[r0 + g + 8][kk + 8 + 2 * t]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c0 = wn * 32 + j * 8;
                b[j][0] = *reinterpret_cast<const unsigned*>(&Bs[c0 + g][kk + 2 * t]);
                b[j][1] = *reinterpret_cast<const unsigned*>(&Bs[c0 + g][kk + 8 + 2 * t]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i][0], a[i][1], a[i][2], a[i][3], b[j][0], b[j][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = m0 + wm * 32 + i * 16 + g + (r >= 2 ? 8 : 0);
                const int col = n0 + wn * 32 + j * 8 + 2 * t + (r & 1);
                if (row >= M || col >= N) continue;
                float v = acc[i][j][r] + (bias ? bias[col] : 0.f);
                if (EPI == EPI_TANH) v = tanhf(v);
                if (EPI == EPI_DTANH) {
                    const float h = aux[(long long)row * ldc + col];
                    v *= 1.f - h * h;
                }
                C[(long long)row * ldc + col] = v;
            }
}

// dY = 2 (Y - T) / (n n_out); per-block partial sums of (Y - T)^2
__global__ void k_loss(long long total, float scale, const float* __restrict__ Y, const float* __restrict__ T,
                       float* __restrict__ dY, double* __restrict__ partial) {
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const float d = Y[i] - T[i];
        dY[i] = 2.f * d * scale;
        s += (double)d * d;
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) partial[blockIdx.x] = s;
    }
}

// db[c] = sum_m dZ[m][c] (one thread per column, fixed order)
__global__ void k_colsum(int n, int cols, const float* __restrict__ dZ, float* __restrict__ db) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int m = 0; m < n; ++m) s += dZ[(long long)m * cols + c];
    db[c] = s;
}

__global__ void k_adam(int P, float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

}  // namespace

struct fbim_mlp_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    int max_batch = 0;
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    float* h[kLayers] = {nullptr, nullptr, nullptr, nullptr};  // h[1..3]: hidden activations
    float *y = nullptr, *dz0 = nullptr, *dz1 = nullptr;
    double* partial = nullptr;
    long long t = 0;
    long long launches = 0;
    float in_shift[6] = {0, 0, 0, 0, 0, 0}, in_scale[6] = {1, 1, 1, 1, 1, 1};
    float out_scale[36];
    std::string err;
};

namespace fbim {

// Forward pass on n <= max_batch inputs X [n][6] (device); output in mlp->y [n][36].
fbim_status mlp_forward(fbim_mlp_s* P, int n, const float* X) {
    const float* in = X;
    for (int l = 0; l < kLayers; ++l) {
        const int n_in = kWidth[l], n_out = kWidth[l + 1];
        const float* W = P->theta + param_offset_W(l);
        const float* b = P->theta + param_offset_b(l);
        float* out = l < kLayers - 1 ? P->h[l + 1] : P->y;
        dim3 grid((n_out + BN - 1) / BN, (n + BM - 1) / BM);
        if (l < kLayers - 1)
            k_gemm_bf16<EPI_TANH><<<grid, 128, 0, P->stream>>>(n, n_out, n_in, in, n_in, 1, W, 1, n_in, b, nullptr,
                                                              out, n_out);
        else
            k_gemm_bf16<EPI_LINEAR><<<grid, 128, 0, P->stream>>>(n, n_out, n_in, in, n_in, 1, W, 1, n_in, b,
                                                                nullptr, out, n_out);
        ++P->launches;
        in = out;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        P->err = std::string("mlp forward: ") + cudaGetErrorString(e);
        return FBIM_ERR_CUDA;
    }
    return FBIM_OK;
}

const float* mlp_output(const fbim_mlp_s* P) { return P->y; }
const float* mlp_in_shift(const fbim_mlp_s* P) { return P->in_shift; }
const float* mlp_in_scale(const fbim_mlp_s* P) { return P->in_scale; }
const float* mlp_out_scale(const fbim_mlp_s* P) { return P->out_scale; }
int mlp_max_batch(const fbim_mlp_s* P) { return P->max_batch; }
long long* mlp_launch_counter(fbim_mlp_s* P) { return &P->launches; }
void mlp_set_stream(fbim_mlp_s* P, cudaStream_t s) { P->stream = s; }

}  // namespace fbim

namespace {

// Loss and gradient of the whole parameter vector into P->grad; loss to *loss (host).
fbim_status mlp_gradient(fbim_mlp_s* P, int n, const float* X, const float* T, double* loss) {
    FBIM_TRY(fbim::mlp_forward(P, n, X));
    const int n_out = kWidth[kLayers];
    const long long total = (long long)n * n_out;
    const int nb = 120;
    k_loss<<<nb, 256, 0, P->stream>>>(total, 1.f / (float)total, P->y, T, P->dz0, P->partial);
    ++P->launches;
    float* dz = P->dz0;
    float* dz_next = P->dz1;
    for (int l = kLayers - 1; l >= 0; --l) {
        const int n_in = kWidth[l], no = kWidth[l + 1];
        const float* a = l > 0 ? P->h[l] : X;
        float* gW = P->grad + param_offset_W(l);
        float* gb = P->grad + param_offset_b(l);
        // gW [no][n_in] = dZ^T a
        dim3 gw((n_in + BN - 1) / BN, (no + BM - 1) / BM);
        k_gemm_bf16<EPI_LINEAR><<<gw, 128, 0, P->stream>>>(no, n_in, n, dz, 1, no, a, n_in, 1, nullptr, nullptr, gW,
                                                          n_in);
        k_colsum<<<(no + 127) / 128, 128, 0, P->stream>>>(n, no, dz, gb);
        P->launches += 2;
        if (l > 0) {
            // dZ_{l-1} = (dZ W) * (1 - a^2)
            const float* W = P->theta + param_offset_W(l);
            dim3 gx((n_in + BN - 1) / BN, (n + BM - 1) / BM);
            k_gemm_bf16<EPI_DTANH><<<gx, 128, 0, P->stream>>>(n, n_in, no, dz, no, 1, W, n_in, 1, nullptr, a,
                                                             dz_next, n_in);
            ++P->launches;
            std::swap(dz, dz_next);
        }
    }
    std::vector<double> part(nb);
    cudaError_t e = cudaMemcpyAsync(part.data(), P->partial, sizeof(double) * nb, cudaMemcpyDeviceToHost, P->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) {
        P->err = std::string("mlp gradient: ") + cudaGetErrorString(e);
        return FBIM_ERR_CUDA;
    }
    double s = 0.0;
    for (double x : part) s += x;
    if (loss) *loss = s / (double)total;
    return FBIM_OK;
}

bool alloc_f(float** p, size_t n) { return cudaMalloc(p, sizeof(float) * n) == cudaSuccess; }

}  // namespace

extern "C" int fbim_mlp_param_count(void) { return kParams; }

extern "C" void fbim_mlp_destroy(fbim_mlp P) {
    if (!P) return;
    cudaSetDevice(P->device);
    for (float* p : {P->theta, P->m, P->v, P->grad, P->h[1], P->h[2], P->h[3], P->y, P->dz0, P->dz1}) cudaFree(p);
    cudaFree(P->partial);
    delete P;
}

extern "C" fbim_status fbim_mlp_create(fbim_mlp* out, int max_batch, void* stream, int device) {
    if (!out || max_batch <= 0 || max_batch > (1 << 24)) return FBIM_ERR_INVALID_ARG;
    *out = nullptr;
    fbim_mlp P = new (std::nothrow) fbim_mlp_s();
    if (!P) return FBIM_ERR_OOM;
    P->device = device;
    P->stream = (cudaStream_t)stream;
    P->max_batch = max_batch;
    for (float& s : P->out_scale) s = 1.f;
    if (cudaSetDevice(device) != cudaSuccess) {
        delete P;
        return FBIM_ERR_CUDA;
    }
    const size_t mb = (size_t)max_batch;
    bool ok = alloc_f(&P->theta, kParams) && alloc_f(&P->m, kParams) && alloc_f(&P->v, kParams) &&
              alloc_f(&P->grad, kParams) && alloc_f(&P->h[1], mb * 128) && alloc_f(&P->h[2], mb * 128) &&
              alloc_f(&P->h[3], mb * 128) && alloc_f(&P->y, mb * 36) && alloc_f(&P->dz0, mb * 128) &&
              alloc_f(&P->dz1, mb * 128) && cudaMalloc(&P->partial, sizeof(double) * 120) == cudaSuccess;
    ok = ok && cudaMemsetAsync(P->theta, 0, sizeof(float) * kParams, P->stream) == cudaSuccess &&
         cudaMemsetAsync(P->m, 0, sizeof(float) * kParams, P->stream) == cudaSuccess &&
         cudaMemsetAsync(P->v, 0, sizeof(float) * kParams, P->stream) == cudaSuccess &&
         cudaStreamSynchronize(P->stream) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        fbim::set_global_error("fbim_mlp_create: device allocation failed");
        fbim_mlp_destroy(P);
        return FBIM_ERR_OOM;
    }
    *out = P;
    return FBIM_OK;
}

extern "C" fbim_status fbim_mlp_set_params(fbim_mlp P, const float* theta_host) {
    if (!P || !theta_host) return FBIM_ERR_INVALID_ARG;
    cudaSetDevice(P->device);
    // a new parameter vector restarts the optimizer
    P->t = 0;
    if (cudaMemcpyAsync(P->theta, theta_host, sizeof(float) * kParams, cudaMemcpyHostToDevice, P->stream) !=
            cudaSuccess ||
        cudaMemsetAsync(P->m, 0, sizeof(float) * kParams, P->stream) != cudaSuccess ||
        cudaMemsetAsync(P->v, 0, sizeof(float) * kParams, P->stream) != cudaSuccess ||
        cudaStreamSynchronize(P->stream) != cudaSuccess) {
        P->err = "fbim_mlp_set_params: copy failed";
        return FBIM_ERR_CUDA;
    }
    return FBIM_OK;
}

extern "C" fbim_status fbim_mlp_get_params(fbim_mlp P, float* theta_host) {
    if (!P || !theta_host) return FBIM_ERR_INVALID_ARG;
    cudaSetDevice(P->device);
    if (cudaMemcpyAsync(theta_host, P->theta, sizeof(float) * kParams, cudaMemcpyDeviceToHost, P->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(P->stream) != cudaSuccess) {
        P->err = "fbim_mlp_get_params: copy failed";
        return FBIM_ERR_CUDA;
    }
    return FBIM_OK;
}

extern "C" fbim_status fbim_mlp_set_normalization(fbim_mlp P, const float* in_shift, const float* in_scale,
                                                  const float* out_scale) {
    if (!P || !in_shift || !in_scale || !out_scale) return FBIM_ERR_INVALID_ARG;
    for (int i = 0; i < 6; ++i)
        if (!(in_scale[i] > 0.f) || !std::isfinite(in_shift[i])) return FBIM_ERR_INVALID_ARG;
    for (int i = 0; i < 36; ++i)
        if (!std::isfinite(out_scale[i])) return FBIM_ERR_INVALID_ARG;
    std::memcpy(P->in_shift, in_shift, sizeof(P->in_shift));
    std::memcpy(P->in_scale, in_scale, sizeof(P->in_scale));
    std::memcpy(P->out_scale, out_scale, sizeof(P->out_scale));
    return FBIM_OK;
}

extern "C" fbim_status fbim_mlp_forward(fbim_mlp P, int n, const float* X_dev, float* Y_dev) {
    if (!P || n < 0 || n > P->max_batch || (n > 0 && (!X_dev || !Y_dev))) return FBIM_ERR_INVALID_ARG;
    if (n == 0) return FBIM_OK;
    cudaSetDevice(P->device);
    FBIM_TRY(fbim::mlp_forward(P, n, X_dev));
    if (cudaMemcpyAsync(Y_dev, P->y, sizeof(float) * 36 * (size_t)n, cudaMemcpyDeviceToDevice, P->stream) !=
        cudaSuccess) {
        P->err = "fbim_mlp_forward: copy failed";
        return FBIM_ERR_CUDA;
    }
    return FBIM_OK;
}

extern "C" fbim_status fbim_mlp_gradient(fbim_mlp P, int n, const float* X_dev, const float* T_dev, float* grad_dev,
                                         double* loss) {
    if (!P || n <= 0 || n > P->max_batch || !X_dev || !T_dev) return FBIM_ERR_INVALID_ARG;
    cudaSetDevice(P->device);
    FBIM_TRY(mlp_gradient(P, n, X_dev, T_dev, loss));
    if (grad_dev && cudaMemcpyAsync(grad_dev, P->grad, sizeof(float) * kParams, cudaMemcpyDeviceToDevice,
                                    P->stream) != cudaSuccess) {
        P->err = "fbim_mlp_gradient: copy failed";
        return FBIM_ERR_CUDA;
    }
    return FBIM_OK;
}

extern "C" fbim_status fbim_mlp_adam_step(fbim_mlp P, int n, const float* X_dev, const float* T_dev, float lr,
                                          float beta1, float beta2, float eps, double* loss) {
    if (!P || n <= 0 || n > P->max_batch || !X_dev || !T_dev || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) ||
        !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
        return FBIM_ERR_INVALID_ARG;
    cudaSetDevice(P->device);
    FBIM_TRY(mlp_gradient(P, n, X_dev, T_dev, loss));
    ++P->t;
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)beta1, (double)P->t)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)beta2, (double)P->t)));
    k_adam<<<(kParams + 255) / 256, 256, 0, P->stream>>>(kParams, P->theta, P->m, P->v, P->grad, lr, beta1, beta2,
                                                          eps, c1, c2);
    ++P->launches;
    if (cudaGetLastError() != cudaSuccess) {
        P->err = "fbim_mlp_adam_step: launch failed";
        return FBIM_ERR_CUDA;
    }
    return FBIM_OK;
}

extern "C" long long fbim_mlp_launches(fbim_mlp P) { return P ? P->launches : 0; }

extern "C" const char* fbim_mlp_last_error(fbim_mlp P) { return P ? P->err.c_str() : fbim::global_error(); }
