// Learned coarse level on top of the block-diagonal preconditioner (Sec. 3.4,
// Eq. preconditionerGMRES).  The block preconditioner solves each body alone:
// with g = M_bb^+ r_mu and the effective force a_b = r_U,b + K_b^T g_b, it sets
// U_b = -N~_b a_b and mu_b = g_b + M_bb^+ K_b U_b.  The coarse level adds the
// hydrodynamic coupling of close pairs to the body mobilities:
//   U_b = -N~_b a_b - sum over close pairs (p, q) containing b of (C_pq [a_p; a_q])_b,
// with C_pq a 6x6 pair-mobility correction predicted by the pair network from the
// pair's geometry, and mu_b recomputed from that U_b.
//
// Setup, at every new configuration: candidate pairs by centre distance (below
// twice the body radius plus g_c), their gap (smallest node-to-node distance,
// minimum image), the close pairs (gap < g_c, alpha-major), their features, the
// network, and C in the lab frame, T(theta_a) C T(theta_a)^T.  A pair's C is
// dropped when blockdiag(N~_p, N~_q) + C_pq is not positive definite or not
// finite.  Setup reads two counts back to the host; the application kernels are
// stream-ordered and sized by buffer capacity (the live pair count is read on the
// device), so captured graphs stay valid while the capacity holds.
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "fbim_internal.h"
#include "solver.cuh"

namespace fbim {
fbim_status mlp_forward(fbim_mlp_s* P, int n, const float* X);
const float* mlp_output(const fbim_mlp_s* P);
const float* mlp_in_shift(const fbim_mlp_s* P);
const float* mlp_in_scale(const fbim_mlp_s* P);
const float* mlp_out_scale(const fbim_mlp_s* P);
int mlp_max_batch(const fbim_mlp_s* P);
void mlp_set_stream(fbim_mlp_s* P, cudaStream_t s);
}  // namespace fbim

struct Coarse {
    fbim_mlp_s* model = nullptr;
    double g_c = 0, r_env = 0;
    unsigned long long geom_seen = ~0ull;
    int n_pairs = 0, n_rejected = 0;
    int cap_cand = 0, cap_pairs = 0;
    int* cand_count = nullptr;   // [n_b] candidates per body
    int* cand_start = nullptr;   // [scan_storage(n_b)] exclusive scan (n_b + 1 used)
    int2* cand = nullptr;        // [cap_cand] (a, b), a-major
    double* cand_gap = nullptr;  // [cap_cand]
    int* keep = nullptr;         // [cap_cand] gap < g_c
    int* keep_idx = nullptr;     // [scan_storage(cap_cand)]
    int* first_start = nullptr;  // [n_b + 1] pairs whose first body is b: [first_start[b], first_start[b+1])
    int2* pairs = nullptr;       // [cap_pairs]
    double* feat = nullptr;      // [cap_pairs][6] raw features
    float* xin = nullptr;        // [cap_pairs][6] normalised features
    float* y = nullptr;          // [cap_pairs][36] network output
    double* C = nullptr;         // [cap_pairs][36] lab-frame corrections, row-major 6 x 6
    int* sec_count = nullptr;    // [n_b] pairs whose second body is b
    int* sec_start = nullptr;    // [scan_storage(n_b)]
    int* sec_fill = nullptr;     // [n_b]
    int* sec_list = nullptr;     // [cap_pairs]
    double* a_lab = nullptr;     // [n_b][3] effective body forces (lab frame)
    double* U_bd = nullptr;      // [n_b][3] block-diagonal velocities (lab frame)
    double* dU = nullptr;        // [cap_pairs][6] pair contributions
    int* d_n_pairs = nullptr;    // [1] live pair count
    int* d_rejected = nullptr;   // [1]
};

namespace {

struct Norm6 {
    float shift[6], scale[6];
};
struct Scale36 {
    float s[36];
};

__device__ __forceinline__ double wrap(double d, double L) { return d - L * rint(d / L); }

__global__ void k_cand_count(int n_b, const double* __restrict__ Q, double L, double reach2, int* __restrict__ cnt) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_b) return;
    const double xa = Q[3 * a], ya = Q[3 * a + 1];
    int c = 0;
    for (int b = a + 1; b < n_b; ++b) {
        const double dx = wrap(Q[3 * b] - xa, L), dy = wrap(Q[3 * b + 1] - ya, L);
        c += (dx * dx + dy * dy < reach2) ? 1 : 0;
    }
    cnt[a] = c;
}

__global__ void k_cand_fill(int n_b, const double* __restrict__ Q, double L, double reach2,
                            const int* __restrict__ start, int2* __restrict__ cand) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_b) return;
    const double xa = Q[3 * a], ya = Q[3 * a + 1];
    int o = start[a];
    for (int b = a + 1; b < n_b; ++b) {
        const double dx = wrap(Q[3 * b] - xa, L), dy = wrap(Q[3 * b + 1] - ya, L);
        if (dx * dx + dy * dy < reach2) cand[o++] = make_int2(a, b);
    }
}

// one warp per candidate: smallest node-to-node distance (minimum image)
__global__ void k_cand_gap(int n_cand, int n_p, const double* __restrict__ x, double L, double g_c,
                           const int2* __restrict__ cand, double* __restrict__ gap, int* __restrict__ keep) {
    const int c = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= n_cand) return;
    const int a = cand[c].x, b = cand[c].y;
    const double* xa = x + 2 * (size_t)a * n_p;
    const double* xb = x + 2 * (size_t)b * n_p;
    double best = 1e300;
    for (int i = lane; i < n_p; i += 32) {
        const double px = xa[2 * i], py = xa[2 * i + 1];
        for (int j = 0; j < n_p; ++j) {
            const double dx = wrap(xb[2 * j] - px, L), dy = wrap(xb[2 * j + 1] - py, L);
            best = fmin(best, dx * dx + dy * dy);
        }
    }
    for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (lane == 0) {
        const double gp = sqrt(best);
        gap[c] = gp;
        keep[c] = gp < g_c ? 1 : 0;
    }
}

__global__ void k_pair_feats(int n_cand, const int2* __restrict__ cand, const int* __restrict__ keep,
                             const int* __restrict__ keep_idx, const double* __restrict__ gap,
                             const double* __restrict__ Q, double L, Norm6 nrm, int2* __restrict__ pairs,
                             double* __restrict__ feat, float* __restrict__ xin) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cand || !keep[c]) return;
    const int p = keep_idx[c];
    const int a = cand[c].x, b = cand[c].y;
    pairs[p] = make_int2(a, b);
    const double dx = wrap(Q[3 * b] - Q[3 * a], L), dy = wrap(Q[3 * b + 1] - Q[3 * a + 1], L);
    double sa, ca;
    sincos(Q[3 * a + 2], &sa, &ca);
    double ph_s, ph_c;
    sincos(Q[3 * b + 2] - Q[3 * a + 2], &ph_s, &ph_c);
    const double f[6] = {ca * dx + sa * dy, -sa * dx + ca * dy, sqrt(dx * dx + dy * dy), ph_c, ph_s, gap[c]};
    for (int k = 0; k < 6; ++k) {
        feat[6 * (size_t)p + k] = f[k];
        xin[6 * (size_t)p + k] = (float)((f[k] - (double)nrm.shift[k]) / (double)nrm.scale[k]);
    }
}

__global__ void k_first_start(int n_b, const int* __restrict__ cand_start, const int* __restrict__ keep_idx,
                              int* __restrict__ first_start) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a <= n_b) first_start[a] = keep_idx[cand_start[a]];
}

// C in the lab frame with the positive-definiteness test of blockdiag(N~_p, N~_q) + C
__global__ void k_pair_C(int n_pairs, const int2* __restrict__ pairs, const double* __restrict__ Q,
                         const float* __restrict__ y, Scale36 os, double n0, double n1, double n2, double n3,
                         double n4, double n5, double n6, double n7, double n8, double* __restrict__ Cout,
                         int* __restrict__ rejected) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs) return;
    const int a = pairs[p].x, b = pairs[p].y;
    double Cf[6][6];
    bool finite = true;
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            const double v = (double)y[36 * (size_t)p + 6 * i + j] * (double)os.s[6 * i + j];
            Cf[i][j] = v;
            finite = finite && isfinite(v);
        }
    double T[6][6] = {};
    double s, c;
    sincos(Q[3 * a + 2], &s, &c);
    for (int blk = 0; blk < 2; ++blk) {
        const int o = 3 * blk;
        T[o][o] = c;
        T[o][o + 1] = -s;
        T[o + 1][o] = s;
        T[o + 1][o + 1] = c;
        T[o + 2][o + 2] = 1.0;
    }
    // Cs = sym(Cf); C = T Cs T^T
    double TC[6][6];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double acc = 0;
            for (int k = 0; k < 6; ++k) acc += T[i][k] * 0.5 * (Cf[k][j] + Cf[j][k]);
            TC[i][j] = acc;
        }
    double C[6][6];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double acc = 0;
            for (int k = 0; k < 6; ++k) acc += TC[i][k] * T[j][k];
            C[i][j] = acc;
        }
    // S = blockdiag(N~_a, N~_b) (lab frame) + C, Cholesky
    const double Nr[3][3] = {{n0, n1, n2}, {n3, n4, n5}, {n6, n7, n8}};
    double S[6][6];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) S[i][j] = C[i][j];
    for (int blk = 0; blk < 2; ++blk) {
        double sb, cb;
        sincos(Q[3 * (blk ? b : a) + 2], &sb, &cb);
        const double R[3][3] = {{cb, -sb, 0}, {sb, cb, 0}, {0, 0, 1}};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) acc += R[i][k] * Nr[k][l] * R[j][l];
                S[3 * blk + i][3 * blk + j] += acc;
            }
    }
    bool spd = finite;
    for (int j = 0; j < 6 && spd; ++j) {
        double d = S[j][j];
        for (int k = 0; k < j; ++k) d -= S[j][k] * S[j][k];
        if (!(d > 0)) {
            spd = false;
            break;
        }
        const double l = sqrt(d);
        S[j][j] = l;
        for (int i = j + 1; i < 6; ++i) {
            double v = S[i][j];
            for (int k = 0; k < j; ++k) v -= S[i][k] * S[j][k];
            S[i][j] = v / l;
        }
    }
    if (!spd) atomicAdd(rejected, 1);
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) Cout[36 * (size_t)p + 6 * i + j] = spd ? C[i][j] : 0.0;
}

__global__ void k_sec_count(int n_pairs, const int2* __restrict__ pairs, int* __restrict__ cnt) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n_pairs) atomicAdd(&cnt[pairs[p].y], 1);
}

__global__ void k_sec_fill(int n_pairs, const int2* __restrict__ pairs, const int* __restrict__ start,
                           int* __restrict__ fill, int* __restrict__ list) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs) return;
    const int b = pairs[p].y;
    list[start[b] + atomicAdd(&fill[b], 1)] = p;
}

}  // namespace

namespace {

// Per body: effective force a = R (R^T r_U + K_ref^T g) and the block-diagonal
// velocity U_bd = -R N~ (R^T r_U + K_ref^T g), both in the lab frame.
template <typename T>
__global__ void k_coarse_a(int n_p, const double* __restrict__ ref, const double* __restrict__ rot,
                           const T* __restrict__ g, const double* __restrict__ rU, double n0, double n1, double n2,
                           double n3, double n4, double n5, double n6, double n7, double n8,
                           double* __restrict__ a_lab, double* __restrict__ U_bd) {
    const int b = blockIdx.x;
    const T* gb = g + (size_t)b * 2 * n_p;
    double sx = 0, sy = 0, st = 0;
    for (int j = threadIdx.x; j < n_p; j += blockDim.x) {
        const double gx = (double)gb[2 * j], gy = (double)gb[2 * j + 1];
        sx += gx;
        sy += gy;
        st += ref[2 * j] * gy - ref[2 * j + 1] * gx;
    }
    __shared__ double red[3][32];
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
    if (threadIdx.x == 0) {
        double tx = 0, ty = 0, tt = 0;
        for (int w = 0; w < nw; ++w) {
            tx += red[0][w];
            ty += red[1][w];
            tt += red[2][w];
        }
        const double c = rot[2 * b], s = rot[2 * b + 1];
        const double ax = c * rU[3 * b] + s * rU[3 * b + 1] + tx;
        const double ay = -s * rU[3 * b] + c * rU[3 * b + 1] + ty;
        const double at = rU[3 * b + 2] + tt;
        a_lab[3 * b] = c * ax - s * ay;
        a_lab[3 * b + 1] = s * ax + c * ay;
        a_lab[3 * b + 2] = at;
        const double u0 = -(n0 * ax + n1 * ay + n2 * at);
        const double u1 = -(n3 * ax + n4 * ay + n5 * at);
        const double u2 = -(n6 * ax + n7 * ay + n8 * at);
        U_bd[3 * b] = c * u0 - s * u1;
        U_bd[3 * b + 1] = s * u0 + c * u1;
        U_bd[3 * b + 2] = u2;
    }
}

// dU_p = -C_p [a_first; a_second] for the live pairs
__global__ void k_coarse_pairs(int cap, const int* __restrict__ n_live, const int2* __restrict__ pairs,
                               const double* __restrict__ C, const double* __restrict__ a_lab,
                               double* __restrict__ dU) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= cap || p >= *n_live) return;
    const int a = pairs[p].x, b = pairs[p].y;
    const double v[6] = {a_lab[3 * a], a_lab[3 * a + 1], a_lab[3 * a + 2],
                         a_lab[3 * b], a_lab[3 * b + 1], a_lab[3 * b + 2]};
    const double* Cp = C + 36 * (size_t)p;
    for (int i = 0; i < 6; ++i) {
        double acc = 0;
        for (int k = 0; k < 6; ++k) acc += Cp[6 * i + k] * v[k];
        dU[6 * (size_t)p + i] = -acc;
    }
}

// Per body: U = U_bd + its pair contributions (in pair order), then the traction
// mu = R (g + H R^T U) as in the block solve.
template <typename T>
__global__ void k_coarse_finish(int n_p, const double* __restrict__ rot, const T* __restrict__ g,
                                const T* __restrict__ H, const int* __restrict__ first_start,
                                const int* __restrict__ sec_start, const int* __restrict__ sec_list,
                                const double* __restrict__ dU, const double* __restrict__ U_bd,
                                double* __restrict__ out_mu, double* __restrict__ out_U) {
    const int b = blockIdx.x;
    const int n2 = 2 * n_p;
    __shared__ double Up[3];
    const double c = rot[2 * b], s = rot[2 * b + 1];
    if (threadIdx.x == 0) {
        double U[3] = {U_bd[3 * b], U_bd[3 * b + 1], U_bd[3 * b + 2]};
        for (int p = first_start[b]; p < first_start[b + 1]; ++p)
            for (int k = 0; k < 3; ++k) U[k] += dU[6 * (size_t)p + k];
        // pairs where b is the second body, summed in increasing pair index
        const int s0 = sec_start[b], len = sec_start[b + 1] - s0;
        int idx[32];
        const int n_sorted = len < 32 ? len : 32;
        for (int i = 0; i < n_sorted; ++i) {
            const int v = sec_list[s0 + i];
            int j = i;
            while (j > 0 && idx[j - 1] > v) {
                idx[j] = idx[j - 1];
                --j;
            }
            idx[j] = v;
        }
        for (int i = 0; i < len; ++i) {
            const int p = i < n_sorted ? idx[i] : sec_list[s0 + i];
            for (int k = 0; k < 3; ++k) U[k] += dU[6 * (size_t)p + 3 + k];
        }
        out_U[3 * b] = U[0];
        out_U[3 * b + 1] = U[1];
        out_U[3 * b + 2] = U[2];
        Up[0] = c * U[0] + s * U[1];
        Up[1] = -s * U[0] + c * U[1];
        Up[2] = U[2];
    }
    __syncthreads();
    const T* gb = g + (size_t)b * n2;
    const double u0 = Up[0], u1 = Up[1], u2 = Up[2];
    for (int i = threadIdx.x; i < n_p; i += blockDim.x) {
        const double mx = (double)gb[2 * i] + (double)H[2 * i] * u0 + (double)H[n2 + 2 * i] * u1 +
                          (double)H[2 * n2 + 2 * i] * u2;
        const double my = (double)gb[2 * i + 1] + (double)H[2 * i + 1] * u0 + (double)H[n2 + 2 * i + 1] * u1 +
                          (double)H[2 * n2 + 2 * i + 1] * u2;
        const size_t m = (size_t)b * n_p + i;
        out_mu[2 * m] = c * mx - s * my;
        out_mu[2 * m + 1] = s * mx + c * my;
    }
}

}  // namespace

namespace fbim {

static void free_coarse_buffers(Coarse* C) {
    for (void* p : {(void*)C->cand_count, (void*)C->cand_start, (void*)C->cand, (void*)C->cand_gap, (void*)C->keep,
                    (void*)C->keep_idx, (void*)C->first_start, (void*)C->pairs, (void*)C->feat, (void*)C->xin,
                    (void*)C->y, (void*)C->C, (void*)C->sec_count, (void*)C->sec_start, (void*)C->sec_fill,
                    (void*)C->sec_list, (void*)C->a_lab, (void*)C->U_bd, (void*)C->dU, (void*)C->d_n_pairs,
                    (void*)C->d_rejected})
        cudaFree(p);
}

void free_coarse(fbim_handle_s* h) {
    Coarse* C = h->coarse;
    if (!C) return;
    free_coarse_buffers(C);
    delete C;
    h->coarse = nullptr;
}

// Pair list, features and (with a model) the corrections of the current configuration.
static fbim_status coarse_pairs_setup(fbim_handle_s* h, Coarse* C, bool with_model) {
    const int n_b = h->n_b, tb = 256;
    cudaStream_t st = h->stream;
    const double reach = 2.0 * C->r_env + C->g_c;
    k_cand_count<<<(n_b + tb - 1) / tb, tb, 0, st>>>(n_b, h->Q, h->L, reach * reach, C->cand_count);
    scan_exclusive(st, C->cand_count, n_b, C->cand_start);
    int n_cand = 0;
    FBIM_CUDA_TRY(h, cudaMemcpyAsync(&n_cand, C->cand_start + n_b, sizeof(int), cudaMemcpyDeviceToHost, st));
    FBIM_CUDA_TRY(h, cudaStreamSynchronize(st));
    if (n_cand > C->cap_cand) {
        const int cap = n_cand + n_cand / 4 + 16;
        for (void* p : {(void*)C->cand, (void*)C->cand_gap, (void*)C->keep, (void*)C->keep_idx}) cudaFree(p);
        const bool ok = cudaMalloc(&C->cand, sizeof(int2) * cap) == cudaSuccess &&
                        cudaMalloc(&C->cand_gap, sizeof(double) * cap) == cudaSuccess &&
                        cudaMalloc(&C->keep, sizeof(int) * cap) == cudaSuccess &&
                        cudaMalloc(&C->keep_idx, sizeof(int) * scan_storage(cap)) == cudaSuccess;
        if (!ok) {
            h->fail("coarse level: device allocation failed");
            return FBIM_ERR_OOM;
        }
        C->cap_cand = cap;
    }
    if (!C->keep_idx && cudaMalloc(&C->keep_idx, sizeof(int) * scan_storage(1)) != cudaSuccess) {
        h->fail("coarse level: device allocation failed");
        return FBIM_ERR_OOM;
    }
    int n_pairs = 0;
    if (n_cand > 0) {
        k_cand_fill<<<(n_b + tb - 1) / tb, tb, 0, st>>>(n_b, h->Q, h->L, reach * reach, C->cand_start, C->cand);
        k_cand_gap<<<(unsigned)(((size_t)n_cand * 32 + 255) / 256), 256, 0, st>>>(
            n_cand, h->n_p, h->x, h->L, C->g_c, C->cand, C->cand_gap, C->keep);
        scan_exclusive(st, C->keep, n_cand, C->keep_idx);
        h->launches += 2;
        FBIM_CUDA_TRY(h, cudaMemcpyAsync(&n_pairs, C->keep_idx + n_cand, sizeof(int), cudaMemcpyDeviceToHost, st));
        FBIM_CUDA_TRY(h, cudaStreamSynchronize(st));
    } else {
        FBIM_CUDA_TRY(h, cudaMemsetAsync(C->keep_idx, 0, sizeof(int), st));
    }
    h->launches += 1;
    const int need = std::max(n_pairs, 1);
    if (need > C->cap_pairs) {
        const int cap = need + need / 4 + 16;
        for (void* p : {(void*)C->pairs, (void*)C->feat, (void*)C->xin, (void*)C->y, (void*)C->C, (void*)C->sec_list,
                        (void*)C->dU})
            cudaFree(p);
        const bool ok = cudaMalloc(&C->pairs, sizeof(int2) * cap) == cudaSuccess &&
                        cudaMalloc(&C->feat, sizeof(double) * 6 * cap) == cudaSuccess &&
                        cudaMalloc(&C->xin, sizeof(float) * 6 * cap) == cudaSuccess &&
                        cudaMalloc(&C->y, sizeof(float) * 36 * cap) == cudaSuccess &&
                        cudaMalloc(&C->C, sizeof(double) * 36 * cap) == cudaSuccess &&
                        cudaMalloc(&C->sec_list, sizeof(int) * cap) == cudaSuccess &&
                        cudaMalloc(&C->dU, sizeof(double) * 6 * cap) == cudaSuccess;
        if (!ok) {
            h->fail("coarse level: device allocation failed");
            return FBIM_ERR_OOM;
        }
        C->cap_pairs = cap;
        ++h->layout_version;  // captured launches hold these pointers and the capacity
    }
    Norm6 nrm;
    for (int k = 0; k < 6; ++k) {
        nrm.shift[k] = C->model ? mlp_in_shift(C->model)[k] : 0.f;
        nrm.scale[k] = C->model ? mlp_in_scale(C->model)[k] : 1.f;
    }
    if (n_cand > 0) {
        k_pair_feats<<<(n_cand + tb - 1) / tb, tb, 0, st>>>(n_cand, C->cand, C->keep, C->keep_idx, C->cand_gap, h->Q,
                                                           h->L, nrm, C->pairs, C->feat, C->xin);
        k_first_start<<<(n_b + 1 + tb - 1) / tb, tb, 0, st>>>(n_b, C->cand_start, C->keep_idx, C->first_start);
        h->launches += 2;
    } else {
        FBIM_CUDA_TRY(h, cudaMemsetAsync(C->first_start, 0, sizeof(int) * (n_b + 1), st));
    }
    C->n_pairs = n_pairs;
    C->n_rejected = 0;
    FBIM_CUDA_TRY(h, cudaMemcpyAsync(C->d_n_pairs, &C->n_pairs, sizeof(int), cudaMemcpyHostToDevice, st));
    FBIM_CUDA_TRY(h, cudaMemsetAsync(C->d_rejected, 0, sizeof(int), st));
    FBIM_CUDA_TRY(h, cudaMemsetAsync(C->sec_count, 0, sizeof(int) * n_b, st));
    FBIM_CUDA_TRY(h, cudaMemsetAsync(C->sec_fill, 0, sizeof(int) * n_b, st));
    if (n_pairs > 0) {
        k_sec_count<<<(n_pairs + tb - 1) / tb, tb, 0, st>>>(n_pairs, C->pairs, C->sec_count);
        h->launches += 1;
    }
    scan_exclusive(st, C->sec_count, n_b, C->sec_start);
    h->launches += 1;
    if (n_pairs > 0) {
        k_sec_fill<<<(n_pairs + tb - 1) / tb, tb, 0, st>>>(n_pairs, C->pairs, C->sec_start, C->sec_fill, C->sec_list);
        h->launches += 1;
    }
    if (with_model && n_pairs > 0) {
        mlp_set_stream(C->model, st);
        const int mb = mlp_max_batch(C->model);
        for (int o = 0; o < n_pairs; o += mb) {
            const int n = std::min(mb, n_pairs - o);
            FBIM_TRY(mlp_forward(C->model, n, C->xin + 6 * (size_t)o));
            FBIM_CUDA_TRY(h, cudaMemcpyAsync(C->y + 36 * (size_t)o, mlp_output(C->model), sizeof(float) * 36 * n,
                                             cudaMemcpyDeviceToDevice, st));
        }
        Scale36 os;
        for (int k = 0; k < 36; ++k) os.s[k] = mlp_out_scale(C->model)[k];
        const double* Nt = h->solver->Nt;
        k_pair_C<<<(n_pairs + tb - 1) / tb, tb, 0, st>>>(n_pairs, C->pairs, h->Q, C->y, os, Nt[0], Nt[1], Nt[2],
                                                         Nt[3], Nt[4], Nt[5], Nt[6], Nt[7], Nt[8], C->C,
                                                         C->d_rejected);
        h->launches += 1;
        FBIM_CUDA_TRY(h, cudaMemcpyAsync(&C->n_rejected, C->d_rejected, sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    FBIM_CUDA_TRY(h, cudaGetLastError());
    FBIM_CUDA_TRY(h, cudaStreamSynchronize(st));
    return FBIM_OK;
}

static fbim_status coarse_alloc(fbim_handle_s* h, Coarse* C) {
    const int n_b = h->n_b;
    const size_t sb = scan_storage(n_b);
    const bool ok = cudaMalloc(&C->cand_count, sizeof(int) * n_b) == cudaSuccess &&
                    cudaMalloc(&C->cand_start, sizeof(int) * sb) == cudaSuccess &&
                    cudaMalloc(&C->first_start, sizeof(int) * (n_b + 1)) == cudaSuccess &&
                    cudaMalloc(&C->sec_count, sizeof(int) * n_b) == cudaSuccess &&
                    cudaMalloc(&C->sec_start, sizeof(int) * sb) == cudaSuccess &&
                    cudaMalloc(&C->sec_fill, sizeof(int) * n_b) == cudaSuccess &&
                    cudaMalloc(&C->a_lab, sizeof(double) * 3 * n_b) == cudaSuccess &&
                    cudaMalloc(&C->U_bd, sizeof(double) * 3 * n_b) == cudaSuccess &&
                    cudaMalloc(&C->d_n_pairs, sizeof(int)) == cudaSuccess &&
                    cudaMalloc(&C->d_rejected, sizeof(int)) == cudaSuccess;
    if (!ok) {
        h->fail("coarse level: device allocation failed");
        return FBIM_ERR_OOM;
    }
    double r = 0;
    for (int j = 0; j < h->n_p; ++j) r = std::max(r, std::hypot(h->host_ref[2 * j], h->host_ref[2 * j + 1]));
    C->r_env = r;
    return FBIM_OK;
}

fbim_status coarse_refresh(fbim_handle_s* h) {
    Coarse* C = h->coarse;
    if (!C || C->geom_seen == h->geom_version) return FBIM_OK;
    FBIM_TRY(ensure_solver(h));
    FBIM_TRY(coarse_pairs_setup(h, C, true));
    C->geom_seen = h->geom_version;
    return FBIM_OK;
}

bool coarse_active(fbim_handle_s* h, fbim_status* st) {
    if (!h->coarse || h->coarse_suspended_geom == h->geom_version) return false;
    *st = coarse_refresh(h);
    return *st == FBIM_OK;
}

template <typename T>
fbim_status coarse_body_solve(fbim_handle_s* h, const T* g, const T* H, const double* rU, double* out_mu,
                              double* out_U) {
    Coarse* C = h->coarse;
    const double* Nt = h->solver->Nt;
    k_coarse_a<T><<<h->n_b, 128, 0, h->stream>>>(h->n_p, h->ref, h->rot, g, rU, Nt[0], Nt[1], Nt[2], Nt[3], Nt[4],
                                                 Nt[5], Nt[6], Nt[7], Nt[8], C->a_lab, C->U_bd);
    k_coarse_pairs<<<(C->cap_pairs + 127) / 128, 128, 0, h->stream>>>(C->cap_pairs, C->d_n_pairs, C->pairs, C->C,
                                                                      C->a_lab, C->dU);
    k_coarse_finish<T><<<h->n_b, 128, 0, h->stream>>>(h->n_p, h->rot, g, H, C->first_start, C->sec_start,
                                                      C->sec_list, C->dU, C->U_bd, out_mu, out_U);
    h->launches += 3;
    return FBIM_OK;
}

template fbim_status coarse_body_solve<float>(fbim_handle_s*, const float*, const float*, const double*, double*,
                                              double*);
template fbim_status coarse_body_solve<double>(fbim_handle_s*, const double*, const double*, const double*, double*,
                                               double*);

}  // namespace fbim

extern "C" fbim_status fbim_coarse_enable(fbim_handle h, fbim_mlp model, double g_c) {
    if (!h || (model && !(g_c > 0))) return FBIM_ERR_INVALID_ARG;
    try {
        if (cudaSetDevice(h->device) != cudaSuccess) return FBIM_ERR_CUDA;
        fbim::free_coarse(h);
        ++h->layout_version;
        if (!model) return FBIM_OK;
        Coarse* C = new (std::nothrow) Coarse();
        if (!C) return FBIM_ERR_OOM;
        h->coarse = C;
        C->model = model;
        C->g_c = g_c;
        fbim_status st = fbim::coarse_alloc(h, C);
        if (st == FBIM_OK) st = fbim::coarse_refresh(h);
        if (st != FBIM_OK) fbim::free_coarse(h);
        return st;
    } catch (...) {
        h->fail("unexpected host exception in fbim_coarse_enable");
        return FBIM_ERR_SETUP;
    }
}

extern "C" fbim_status fbim_coarse_stats(fbim_handle h, int* n_pairs, int* n_rejected) {
    if (!h) return FBIM_ERR_INVALID_ARG;
    if (n_pairs) *n_pairs = h->coarse ? h->coarse->n_pairs : 0;
    if (n_rejected) *n_rejected = h->coarse ? h->coarse->n_rejected : 0;
    return FBIM_OK;
}

extern "C" fbim_status fbim_coarse_pairs(fbim_handle h, double g_c, int max_pairs, int* pairs_dev, double* feat_dev,
                                         int* n_pairs) {
    if (!h || !(g_c > 0) || max_pairs < 0 || !n_pairs) return FBIM_ERR_INVALID_ARG;
    try {
        if (cudaSetDevice(h->device) != cudaSuccess) return FBIM_ERR_CUDA;
        Coarse tmp;  // scratch pair search: no captured launch uses its buffers
        tmp.g_c = g_c;
        const unsigned long long lv = h->layout_version;
        fbim_status st = fbim::coarse_alloc(h, &tmp);
        if (st == FBIM_OK) st = fbim::coarse_pairs_setup(h, &tmp, false);
        h->layout_version = lv;
        if (st == FBIM_OK) {
            *n_pairs = tmp.n_pairs;
            const int n = std::min(tmp.n_pairs, max_pairs);
            if (n > 0 && pairs_dev &&
                cudaMemcpyAsync(pairs_dev, tmp.pairs, sizeof(int2) * n, cudaMemcpyDeviceToDevice, h->stream) !=
                    cudaSuccess)
                st = FBIM_ERR_CUDA;
            if (st == FBIM_OK && n > 0 && feat_dev &&
                cudaMemcpyAsync(feat_dev, tmp.feat, sizeof(double) * 6 * n, cudaMemcpyDeviceToDevice, h->stream) !=
                    cudaSuccess)
                st = FBIM_ERR_CUDA;
            if (st == FBIM_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) st = FBIM_ERR_CUDA;
        }
        fbim::free_coarse_buffers(&tmp);
        return st;
    } catch (...) {
        h->fail("unexpected host exception in fbim_coarse_pairs");
        return FBIM_ERR_SETUP;
    }
}
