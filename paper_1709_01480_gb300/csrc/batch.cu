// Batched mobility solves: many independent suspensions, each with any number
// of right-hand sides, solved together (the batched form of the first-kind
// saddle system of Sec. 3.1 with the block-diagonal preconditioner of Sec. 3.4).
//
// Every (handle, right-hand side) pair is one system; the systems are stacked
// into one long FP64 vector.  A Krylov step applies the preconditioner and the
// saddle operator of ALL systems by replaying one captured CUDA graph: for
// each handle the graph holds a branch with the preconditioner GEMM and
// kernels and the whole Ewald matvec (gather, spread, cuFFT, Fourier scale,
// inverse cuFFT, interpolation, pair SpMV, Alpert band and K) of each of its
// right-hand sides in turn.  Branches of different handles share no buffers,
// so the GPU runs them concurrently.  Orthogonalisation (classical
// Gram-Schmidt, twice), norms and updates are segmented kernels over all
// systems at once; the small Hessenberg least-squares problems (Givens
// rotations) run on the host.  Each system stops on its own relative residual;
// its later Krylov vectors are zero, which freezes it.
//
// FBIM_FP32 handles refine: FP64 residuals from a graph of FP64 saddle
// operators and FP32-operator corrections to 1e-4 (one restart cycle each),
// which is the mixed-precision scheme of the single-system solver.
#include <cublas_v2.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "fbim_internal.h"
#include "solver.cuh"

struct fbim_batch_s {
    int n_h = 0, n_tot = 0;                  // handles, systems
    std::vector<fbim_handle> hs;
    std::vector<int> rhs;                    // [n_h] right-hand sides per handle
    std::vector<long long> off;              // [n_tot + 1] system offsets in the stacked vector
    std::vector<int> h_of;                   // [n_tot] handle of each system
    std::vector<long long> f_off, s_off;     // [n_tot] offsets into the caller's stacked F/U and slip arrays
    long long n_all = 0, ld = 0;
    int m = 0;                               // restart length
    int device = 0;
    cudaStream_t stream = nullptr;           // the handles' common stream
    cudaStream_t cap = nullptr;              // origin of the captures (the handles' stream may be the
                                             // legacy default stream, which cannot be captured)
    std::vector<cudaStream_t> side;          // capture branches
    std::vector<cudaEvent_t> side_ev;
    cudaEvent_t fork_ev = nullptr;
    double *V = nullptr, *Z = nullptr, *w = nullptr, *b = nullptr, *x = nullptr, *r = nullptr, *d = nullptr;
    double *vin = nullptr, *zout = nullptr, *wout = nullptr;
    double *dots = nullptr, *hv = nullptr;   // [3][n_tot][m+1] dot products, [n_tot][m+1] scalars
    long long* d_off = nullptr;              // device copy of off
    long long *d_f_off = nullptr, *d_s_off = nullptr;
    int* d_two_n = nullptr;                  // [n_tot] 2N of each system
    // graphs: [0] precondition + saddle FP32, [1] same FP64, [2] saddle FP32, [3] saddle FP64
    cudaGraphExec_t g[4] = {nullptr, nullptr, nullptr, nullptr};
    long long g_kernels[4] = {0, 0, 0, 0};   // this library's kernels in each graph
    std::vector<unsigned long long> g_version[4];
    long long launches = 0;                  // this library's kernels run by the batch (graphs included)
    long long graph_launches = 0;
    std::string err;
};

namespace {

constexpr int kMaxBranches = 64;

// dots[i * stride + j] = <V_j[seg i], w[seg i]>, one block per (i, j).
__global__ void k_seg_dots(const long long* __restrict__ off, const double* __restrict__ V, long long ld,
                           const double* __restrict__ w, double* __restrict__ dots, int stride) {
    const int i = blockIdx.x, j = blockIdx.y;
    const long long a = off[i], e = off[i + 1];
    const double* v = V + (size_t)j * ld;
    double s = 0;
    for (long long t = a + threadIdx.x; t < e; t += blockDim.x) s += v[t] * w[t];
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) dots[(size_t)i * stride + j] = s;
    }
}

__device__ __forceinline__ int seg_of(const long long* __restrict__ off, int n, long long t) {
    int lo = 0, hi = n;  // off[lo] <= t < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= t)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// w[t] -= sum_{j < K} V_j[t] h[seg(t) * stride + j]
__global__ void k_seg_update(long long n_all, const long long* __restrict__ off, int n_seg, int K,
                             const double* __restrict__ V, long long ld, const double* __restrict__ h, int stride,
                             double* __restrict__ w) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_all) return;
    const int i = seg_of(off, n_seg, t);
    double acc = w[t];
    for (int j = 0; j < K; ++j) acc -= V[(size_t)j * ld + t] * h[(size_t)i * stride + j];
    w[t] = acc;
}

// out[t] (+)= sum_{j < K} a[seg(t) * stride + j] in_j[t],  in_j = in + j ld
__global__ void k_seg_combine(long long n_all, const long long* __restrict__ off, int n_seg, int K,
                              const double* __restrict__ a, int stride, const double* in, long long ld,
                              double* out, int accumulate) {  // in may alias out (elementwise)
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_all) return;
    const int i = seg_of(off, n_seg, t);
    double v = accumulate ? out[t] : 0.0;
    for (int j = 0; j < K; ++j) v += a[(size_t)i * stride + j] * in[(size_t)j * ld + t];
    out[t] = v;
}

// w = b - w
__global__ void k_sub(long long n, const double* __restrict__ b, double* __restrict__ w) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) w[t] = b[t] - w[t];
}

// r -= w
__global__ void k_dec(long long n, const double* __restrict__ w, double* __restrict__ r) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) r[t] -= w[t];
}

__global__ void k_add(long long n, const double* __restrict__ d, double* __restrict__ x) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) x[t] += d[t];
}

// stacked right-hand side b = -[slip; F] of every system (zero padding between systems)
__global__ void k_batch_rhs(long long n, const long long* __restrict__ off, int n_seg, const int* __restrict__ two_n,
                            const long long* __restrict__ s_off, const long long* __restrict__ f_off,
                            const double* __restrict__ slip, const double* __restrict__ F, double* __restrict__ b) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int i = seg_of(off, n_seg, t);
    const long long k = t - off[i];
    const int tn = two_n[i];
    const long long len = (long long)tn + (f_off[i + 1] - f_off[i]);
    double v = 0.0;
    if (k < tn)
        v = slip ? -slip[s_off[i] + k] : 0.0;
    else if (k < len)
        v = -F[f_off[i] + (k - tn)];
    b[t] = v;
}

// U of every system from the stacked solution into the caller's stacked [3 n_b] blocks
__global__ void k_batch_u(long long n, const long long* __restrict__ off, int n_seg, const int* __restrict__ two_n,
                          const long long* __restrict__ f_off, const double* __restrict__ x, double* __restrict__ U) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int i = seg_of(off, n_seg, t);
    const long long k = t - off[i] - two_n[i];
    if (k >= 0 && k < f_off[i + 1] - f_off[i]) U[f_off[i] + k] = x[t];
}

fbim_status fail(fbim_batch B, const std::string& m, fbim_status s) {
    B->err = m;
    return s;
}

#define BTRY(expr)                                                                              \
    do {                                                                                        \
        cudaError_t e__ = (expr);                                                               \
        if (e__ != cudaSuccess)                                                                 \
            return fail(B, std::string(#expr) + ": " + cudaGetErrorString(e__), FBIM_ERR_CUDA); \
    } while (0)

#define BSTATUS(expr)                  \
    do {                               \
        fbim_status s__ = (expr);      \
        if (s__ != FBIM_OK) return s__; \
    } while (0)

inline unsigned blocks(long long n, int tb) { return (unsigned)((n + tb - 1) / tb); }

// The operator a graph applies to one system: kind 0/1 = precondition then saddle
// (FP32 / FP64 operator), kind 2/3 = saddle only (FP32 / FP64).
fbim_status system_ops(fbim_batch B, int i, int kind) {
    fbim_handle h = B->hs[B->h_of[i]];
    const bool fp32 = (kind & 1) == 0;
    const double* in = B->vin + B->off[i];
    double* z = B->zout + B->off[i];
    double* y = B->wout + B->off[i];
    if (kind < 2) {
        BSTATUS(fbim::solver_precondition(h, in, z, fp32));
        return fbim::solver_saddle(h, z, y, fp32);
    }
    return fbim::solver_saddle(h, in, y, fp32);
}

bool graph_current(fbim_batch B, int kind) {
    if (!B->g[kind]) return false;
    for (int k = 0; k < B->n_h; ++k)
        if (B->g_version[kind][k] != B->hs[k]->layout_version) return false;
    return true;
}

// Capture graph `kind`: one branch per handle (round-robin over the side
// streams), each running its systems' operators in order.
fbim_status capture(fbim_batch B, int kind) {
    if (graph_current(B, kind)) return FBIM_OK;
    if (B->g[kind]) {
        cudaGraphExecDestroy(B->g[kind]);
        B->g[kind] = nullptr;
    }
    // warm-up outside the capture: first use builds the Ewald buffers, cuFFT plans
    // and the wave-kernel choice, which allocate and synchronise
    std::vector<int> first(B->n_h, -1);
    for (int i = B->n_tot - 1; i >= 0; --i) first[B->h_of[i]] = i;
    for (int k = 0; k < B->n_h; ++k) {
        fbim_status st = system_ops(B, first[k], kind);
        if (st != FBIM_OK) return fail(B, std::string("batch warm-up: ") + B->hs[k]->err, st);
    }
    BTRY(cudaStreamSynchronize(B->stream));
    const int nb = (int)B->side.size();
    std::vector<long long> l0(B->n_h);
    std::vector<bool> timing(B->n_h);
    for (int k = 0; k < B->n_h; ++k) {
        l0[k] = B->hs[k]->launches;
        timing[k] = B->hs[k]->timing;
        B->hs[k]->timing = false;
    }
    cudaGraph_t graph = nullptr;
    BTRY(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
    fbim_status st = FBIM_OK;
    cudaError_t ce = cudaEventRecord(B->fork_ev, B->cap);
    for (int b = 0; b < nb && ce == cudaSuccess; ++b) ce = cudaStreamWaitEvent(B->side[b], B->fork_ev, 0);
    for (int i = 0; i < B->n_tot && st == FBIM_OK && ce == cudaSuccess; ++i) {
        const int k = B->h_of[i];
        fbim::bind_stream(B->hs[k], B->side[k % nb]);
        st = system_ops(B, i, kind);
        if (st != FBIM_OK) B->err = std::string("batch capture: ") + B->hs[k]->err;
    }
    for (int b = 0; b < nb && ce == cudaSuccess; ++b) {
        ce = cudaEventRecord(B->side_ev[b], B->side[b]);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(B->cap, B->side_ev[b], 0);
    }
    const cudaError_t ee = cudaStreamEndCapture(B->cap, &graph);
    long long kernels = 0;
    for (int k = 0; k < B->n_h; ++k) {
        fbim::bind_stream(B->hs[k], B->stream);
        kernels += B->hs[k]->launches - l0[k];
        B->hs[k]->launches = l0[k];  // captured, not run
        B->hs[k]->timing = timing[k];
    }
    if (st != FBIM_OK || ce != cudaSuccess || ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (st != FBIM_OK) return st;
        return fail(B, std::string("batch capture: ") + cudaGetErrorString(ce != cudaSuccess ? ce : ee),
                    FBIM_ERR_CUDA);
    }
    const cudaError_t ie = cudaGraphInstantiate(&B->g[kind], graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        B->g[kind] = nullptr;
        return fail(B, std::string("graph instantiate: ") + cudaGetErrorString(ie), FBIM_ERR_CUDA);
    }
    B->g_kernels[kind] = kernels;
    B->g_version[kind].resize(B->n_h);
    for (int k = 0; k < B->n_h; ++k) B->g_version[kind][k] = B->hs[k]->layout_version;
    return FBIM_OK;
}

// out = op(in) for every system through graph `kind` (in/out: stacked vectors)
fbim_status run_graph(fbim_batch B, int kind, const double* in, double* zout, double* wout) {
    BTRY(cudaMemcpyAsync(B->vin, in, sizeof(double) * B->n_all, cudaMemcpyDeviceToDevice, B->stream));
    BTRY(cudaGraphLaunch(B->g[kind], B->stream));
    if (zout) BTRY(cudaMemcpyAsync(zout, B->zout, sizeof(double) * B->n_all, cudaMemcpyDeviceToDevice, B->stream));
    if (wout) BTRY(cudaMemcpyAsync(wout, B->wout, sizeof(double) * B->n_all, cudaMemcpyDeviceToDevice, B->stream));
    B->launches += B->g_kernels[kind];
    ++B->graph_launches;
    return FBIM_OK;
}

// |v_i|^2 of every system into host vector out (synchronises)
fbim_status seg_norms2(fbim_batch B, const double* v, std::vector<double>& out) {
    const int stride = B->m + 1;
    k_seg_dots<<<dim3(B->n_tot, 1), 256, 0, B->stream>>>(B->d_off, v, 0, v, B->dots, stride);
    B->launches += 1;
    std::vector<double> hc((size_t)B->n_tot * stride);
    BTRY(cudaMemcpyAsync(hc.data(), B->dots, sizeof(double) * hc.size(), cudaMemcpyDeviceToHost, B->stream));
    BTRY(cudaStreamSynchronize(B->stream));
    out.resize(B->n_tot);
    for (int i = 0; i < B->n_tot; ++i) out[i] = hc[(size_t)i * stride];
    return FBIM_OK;
}

// Scale each system's segment of v by s[i] (s on the host), result into out.
fbim_status seg_scale(fbim_batch B, const std::vector<double>& s, const double* v, double* out) {
    BTRY(cudaMemcpyAsync(B->hv, s.data(), sizeof(double) * B->n_tot, cudaMemcpyHostToDevice, B->stream));
    k_seg_combine<<<blocks(B->n_all, 256), 256, 0, B->stream>>>(B->n_all, B->d_off, B->n_tot, 1, B->hv, 1, v, 0,
                                                               out, 0);
    B->launches += 1;
    return FBIM_OK;
}

// Batched right-preconditioned flexible GMRES (restart m, CGS2 Arnoldi) on
// A d = rhs for every system, A through graph `res_kind`, A P through graph
// `op_kind`.  d starts at zero.  System i stops once its residual estimate is
// <= tol[i] |rhs_i|; iters[i] counts its Krylov steps, est[i] its last estimate.
fbim_status batched_fgmres(fbim_batch B, int op_kind, int res_kind, const double* rhs, double* d,
                           const std::vector<double>& tol, int max_iter, std::vector<int>& iters,
                           std::vector<double>& est) {
    const int n = B->n_tot, m = B->m, stride = m + 1;
    const long long N = B->n_all, ld = B->ld;
    const int tb = 256;
    cudaStream_t st = B->stream;
    iters.assign(n, 0);
    est.assign(n, 0.0);
    BTRY(cudaMemsetAsync(d, 0, sizeof(double) * N, st));
    std::vector<double> bn2;
    BSTATUS(seg_norms2(B, rhs, bn2));
    if (op_kind == 0)  // one Gram-Schmidt pass: the second pass's coefficients stay zero
        BTRY(cudaMemsetAsync(B->dots + (size_t)n * stride, 0, sizeof(double) * n * stride, st));
    std::vector<double> bn(n), Hh((size_t)n * m * stride), cs((size_t)n * m), sn((size_t)n * m),
        gv((size_t)n * stride), scale(n), hc((size_t)3 * n * stride), Y((size_t)n * stride);
    for (int i = 0; i < n; ++i) bn[i] = std::sqrt(bn2[i]);
    std::vector<char> active(n);
    std::vector<int> k_used(n);
    int total = 0;
    bool first = true;
    while (true) {
        // w = rhs - A d
        if (first) {
            BTRY(cudaMemcpyAsync(B->w, rhs, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        } else {
            BSTATUS(run_graph(B, res_kind, d, nullptr, B->w));
            k_sub<<<blocks(N, tb), tb, 0, st>>>(N, rhs, B->w);
            B->launches += 1;
        }
        first = false;
        std::vector<double> beta2;
        BSTATUS(seg_norms2(B, B->w, beta2));
        bool any_active = false;
        for (int i = 0; i < n; ++i) {
            const double beta = std::sqrt(beta2[i]);
            if (!std::isfinite(beta)) return fail(B, "batched GMRES residual is not finite", FBIM_ERR_NONFINITE);
            est[i] = bn[i] > 0 ? beta / bn[i] : 0.0;
            active[i] = (bn[i] > 0 && est[i] > tol[i]) ? 1 : 0;
            scale[i] = active[i] ? 1.0 / beta : 0.0;
            std::fill(&gv[(size_t)i * stride], &gv[(size_t)i * stride] + stride, 0.0);
            gv[(size_t)i * stride] = active[i] ? beta : 0.0;
            k_used[i] = 0;
            any_active = any_active || active[i];
        }
        if (!any_active || total >= max_iter) return FBIM_OK;
        BSTATUS(seg_scale(B, scale, B->w, B->V));  // V_0 = w / beta (zero for finished systems)
        int k = 0;
        bool cycle_done = false;
        for (; k < m && total < max_iter && !cycle_done; ++k) {
            BSTATUS(run_graph(B, op_kind, B->V + (size_t)k * ld, B->Z + (size_t)k * ld, B->w));
            // classical Gram-Schmidt: twice with the FP64 operator, once for the FP32-operator
            // corrections of refinement (they stop at ~1e-4; the FP64 residual decides)
            const int passes = op_kind == 0 ? 1 : 2;
            for (int pass = 0; pass < passes; ++pass) {
                double* dst = B->dots + (size_t)pass * n * stride;
                k_seg_dots<<<dim3(n, k + 1), 256, 0, st>>>(B->d_off, B->V, ld, B->w, dst, stride);
                k_seg_update<<<blocks(N, tb), tb, 0, st>>>(N, B->d_off, n, k + 1, B->V, ld, dst, stride, B->w);
            }
            k_seg_dots<<<dim3(n, 1), 256, 0, st>>>(B->d_off, B->w, 0, B->w, B->dots + (size_t)2 * n * stride, stride);
            B->launches += 1 + 2 * passes;
            BTRY(cudaMemcpyAsync(hc.data(), B->dots, sizeof(double) * hc.size(), cudaMemcpyDeviceToHost, st));
            BTRY(cudaStreamSynchronize(st));
            ++total;
            bool any = false;
            for (int i = 0; i < n; ++i) {
                scale[i] = 0.0;
                if (!active[i]) continue;
                const double hn = std::sqrt(hc[(size_t)(2 * n + i) * stride]);
                double* col = &Hh[((size_t)i * m + k) * stride];
                for (int j = 0; j <= k; ++j) col[j] = hc[(size_t)i * stride + j] + hc[(size_t)(n + i) * stride + j];
                col[k + 1] = hn;
                double* c = &cs[(size_t)i * m];
                double* s = &sn[(size_t)i * m];
                double* g = &gv[(size_t)i * stride];
                for (int j = 0; j < k; ++j) {
                    const double t0 = c[j] * col[j] + s[j] * col[j + 1];
                    col[j + 1] = -s[j] * col[j] + c[j] * col[j + 1];
                    col[j] = t0;
                }
                const double den = std::hypot(col[k], col[k + 1]);
                c[k] = den > 0 ? col[k] / den : 1.0;
                s[k] = den > 0 ? col[k + 1] / den : 0.0;
                col[k] = den;
                col[k + 1] = 0.0;
                g[k + 1] = -s[k] * g[k];
                g[k] = c[k] * g[k];
                ++iters[i];
                k_used[i] = k + 1;
                est[i] = std::fabs(g[k + 1]) / bn[i];
                if (!std::isfinite(est[i])) return fail(B, "batched GMRES produced non-finite values",
                                                        FBIM_ERR_NONFINITE);
                if (est[i] <= tol[i] || hn == 0.0) {
                    active[i] = 0;
                } else {
                    scale[i] = 1.0 / hn;
                    any = true;
                }
            }
            if (!any) {
                cycle_done = true;
            } else if (k + 1 < m && total < max_iter) {
                BSTATUS(seg_scale(B, scale, B->w, B->V + (size_t)(k + 1) * ld));
            }
        }
        // d += Z y, y from each system's triangular solve (zero past its k_used)
        std::fill(Y.begin(), Y.end(), 0.0);
        bool all_conv = true;
        for (int i = 0; i < n; ++i) {
            const int ku = k_used[i];
            double* y = &Y[(size_t)i * stride];
            const double* g = &gv[(size_t)i * stride];
            for (int a = ku - 1; a >= 0; --a) {
                double acc = g[a];
                for (int c2 = a + 1; c2 < ku; ++c2) acc -= Hh[((size_t)i * m + c2) * stride + a] * y[c2];
                y[a] = acc / Hh[((size_t)i * m + a) * stride + a];
            }
            all_conv = all_conv && (bn[i] == 0 || est[i] <= tol[i]);
        }
        BTRY(cudaMemcpyAsync(B->hv, Y.data(), sizeof(double) * Y.size(), cudaMemcpyHostToDevice, st));
        k_seg_combine<<<blocks(N, tb), tb, 0, st>>>(N, B->d_off, n, k, B->hv, stride, B->Z, ld, d, 1);
        B->launches += 1;
        BTRY(cudaGetLastError());
        if (all_conv || total >= max_iter) {
            BTRY(cudaStreamSynchronize(st));  // Y (host) must outlive the copy
            return FBIM_OK;
        }
    }
}

// final FP64 relative residual of x for every system
fbim_status final_residual(fbim_batch B, const std::vector<double>& bn, std::vector<double>& rel) {
    BSTATUS(run_graph(B, 3, B->x, nullptr, B->r));
    k_sub<<<blocks(B->n_all, 256), 256, 0, B->stream>>>(B->n_all, B->b, B->r);
    B->launches += 1;
    std::vector<double> rr;
    BSTATUS(seg_norms2(B, B->r, rr));
    rel.resize(B->n_tot);
    for (int i = 0; i < B->n_tot; ++i) rel[i] = bn[i] > 0 ? std::sqrt(rr[i]) / bn[i] : 0.0;
    return FBIM_OK;
}

fbim_status batch_solve(fbim_batch B, const double* F, const double* slip, double tol, int max_iter, double* U,
                        int* iters_out, double* rel_out) {
    const int n = B->n_tot, tb = 256;
    const long long N = B->n_all;
    cudaStream_t st = B->stream;
    const bool fp32 = B->hs[0]->precision == FBIM_FP32;
    // coarse-level pair data of moved handles (host-synchronising: before any capture)
    for (fbim_handle h : B->hs) {
        const fbim_status cs = fbim::coarse_refresh(h);
        if (cs != FBIM_OK) return fail(B, std::string("coarse level: ") + h->err, cs);
    }
    if (fp32) {
        BSTATUS(capture(B, 0));
        BSTATUS(capture(B, 2));
    } else {
        BSTATUS(capture(B, 1));
    }
    BSTATUS(capture(B, 3));
    k_batch_rhs<<<blocks(N, tb), tb, 0, st>>>(N, B->d_off, n, B->d_two_n, B->d_s_off, B->d_f_off, slip, F, B->b);
    B->launches += 1;
    std::vector<double> bn2, bn(n), rel(n, 1.0);
    BSTATUS(seg_norms2(B, B->b, bn2));
    for (int i = 0; i < n; ++i) bn[i] = std::sqrt(bn2[i]);
    std::vector<int> it_tot(n, 0), it;
    std::vector<double> est;
    bool have_rel = false;
    if (!fp32) {
        BSTATUS(batched_fgmres(B, 1, 3, B->b, B->x, std::vector<double>(n, tol), max_iter, it, est));
        it_tot = it;
    } else {
        // iterative refinement (as in the single solve): FP32-operator corrections; the
        // residual is recomputed with the FP64 operators after a correction taken from a
        // residual above 1e-3, else advanced by the inner GMRES's estimate (and, when
        // another correction follows, by r - A_32 d)
        BTRY(cudaMemsetAsync(B->x, 0, sizeof(double) * N, st));
        BTRY(cudaMemcpyAsync(B->r, B->b, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        for (int i = 0; i < n; ++i) rel[i] = bn[i] > 0 ? 1.0 : 0.0;
        std::vector<double> inner(n, 1e-4), keep(n, 1.0);
        int used = 0;
        for (int outer = 0; outer < 40; ++outer) {
            double worst = 0;
            for (int i = 0; i < n; ++i) worst = std::max(worst, rel[i]);
            if (worst <= tol || used >= max_iter) break;
            for (int i = 0; i < n; ++i) {
                // a converged system gets no further correction; the others aim a
                // little below the outer tolerance
                keep[i] = rel[i] <= tol ? 0.0 : 1.0;
                inner[i] = rel[i] > 0 ? std::max(0.3 * tol / rel[i], 1e-4) : 1e-4;
            }
            if (outer > 0) BSTATUS(seg_scale(B, keep, B->r, B->r));
            BSTATUS(batched_fgmres(B, 0, 2, B->r, B->d, inner, std::min(max_iter - used, B->m), it, est));
            int mx = 0;
            double big = 0;
            for (int i = 0; i < n; ++i) {
                it_tot[i] += it[i];
                mx = std::max(mx, it[i]);
                if (keep[i] > 0) big = std::max(big, rel[i]);
            }
            used += std::max(mx, 1);
            k_add<<<blocks(N, tb), tb, 0, st>>>(N, B->d, B->x);
            B->launches += 1;
            if (big > 1e-3) {
                BSTATUS(final_residual(B, bn, rel));
            } else {
                bool more = false;
                for (int i = 0; i < n; ++i) {
                    if (keep[i] > 0) rel[i] *= est[i];
                    more = more || rel[i] > tol;
                }
                if (more && used < max_iter) {
                    BSTATUS(run_graph(B, 2, B->d, nullptr, B->w));
                    k_dec<<<blocks(N, tb), tb, 0, st>>>(N, B->w, B->r);
                    B->launches += 1;
                    std::vector<double> rr;
                    BSTATUS(seg_norms2(B, B->r, rr));
                    for (int i = 0; i < n; ++i)
                        if (keep[i] > 0) rel[i] = bn[i] > 0 ? std::sqrt(rr[i]) / bn[i] : 0.0;
                }
            }
        }
        have_rel = true;
    }
    if (!have_rel) BSTATUS(final_residual(B, bn, rel));
    k_batch_u<<<blocks(N, tb), tb, 0, st>>>(N, B->d_off, n, B->d_two_n, B->d_f_off, B->x, U);
    B->launches += 1;
    BTRY(cudaGetLastError());
    BTRY(cudaStreamSynchronize(st));
    bool conv = true, finite = true;
    for (int i = 0; i < n; ++i) {
        conv = conv && rel[i] <= tol;
        finite = finite && std::isfinite(rel[i]);
        if (iters_out) iters_out[i] = it_tot[i];
        if (rel_out) rel_out[i] = rel[i];
    }
    if (!finite) return fail(B, "batched solve produced non-finite values", FBIM_ERR_NONFINITE);
    if (!conv) return fail(B, "batched GMRES reached the iteration cap before the tolerance", FBIM_ERR_NOT_CONVERGED);
    return FBIM_OK;
}

}  // namespace

extern "C" void fbim_batch_destroy(fbim_batch B) {
    if (!B) return;
    cudaSetDevice(B->device);
    for (double* p : {B->V, B->Z, B->w, B->b, B->x, B->r, B->d, B->vin, B->zout, B->wout, B->dots, B->hv})
        cudaFree(p);
    cudaFree(B->d_off);
    cudaFree(B->d_f_off);
    cudaFree(B->d_s_off);
    cudaFree(B->d_two_n);
    for (cudaGraphExec_t g : B->g)
        if (g) cudaGraphExecDestroy(g);
    for (cudaStream_t s : B->side) cudaStreamDestroy(s);
    for (cudaEvent_t e : B->side_ev) cudaEventDestroy(e);
    if (B->fork_ev) cudaEventDestroy(B->fork_ev);
    if (B->cap) cudaStreamDestroy(B->cap);
    delete B;
}

extern "C" fbim_status fbim_batch_create(fbim_batch* out, int n_handles, const fbim_handle* handles,
                                         const int* n_rhs) {
    if (!out || n_handles <= 0 || !handles) {
        fbim::set_global_error("fbim_batch_create: invalid argument");
        return FBIM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    fbim_batch B = new (std::nothrow) fbim_batch_s();
    if (!B) return FBIM_ERR_OOM;
    try {
        B->n_h = n_handles;
        B->hs.assign(handles, handles + n_handles);
        B->rhs.assign(n_handles, 1);
        for (int k = 0; k < n_handles; ++k) {
            fbim_handle h = B->hs[k];
            if (n_rhs) B->rhs[k] = n_rhs[k];
            if (!h || B->rhs[k] <= 0 || h->stream != B->hs[0]->stream || h->device != B->hs[0]->device ||
                h->precision != B->hs[0]->precision) {
                fbim::set_global_error(
                    "fbim_batch_create: every handle must be valid, have >= 1 right-hand side, and share the "
                    "device, stream and precision of the first");
                delete B;
                return FBIM_ERR_INVALID_ARG;
            }
            for (int j = 0; j < k; ++j)
                if (B->hs[j] == h) {
                    fbim::set_global_error("fbim_batch_create: a handle appears twice (give it more right-hand sides)");
                    delete B;
                    return FBIM_ERR_INVALID_ARG;
                }
        }
        B->device = B->hs[0]->device;
        B->stream = B->hs[0]->stream;
        if (cudaSetDevice(B->device) != cudaSuccess) {
            delete B;
            return FBIM_ERR_CUDA;
        }
        int m = 1 << 30;
        for (auto h : B->hs) {
            const fbim_status st = fbim::ensure_solver(h);
            if (st != FBIM_OK) {
                fbim::set_global_error("fbim_batch_create: " + h->err);
                delete B;
                return st;
            }
            m = std::min(m, h->restart);
        }
        B->m = m;
        for (int k = 0; k < n_handles; ++k) B->n_tot += B->rhs[k];
        const int n = B->n_tot;
        B->off.assign(n + 1, 0);
        B->f_off.assign(n + 1, 0);
        B->s_off.assign(n + 1, 0);
        B->h_of.resize(n);
        std::vector<int> two_n(n);
        for (int k = 0, i = 0; k < n_handles; ++k)
            for (int r = 0; r < B->rhs[k]; ++r, ++i) {
                const fbim_handle h = B->hs[k];
                B->h_of[i] = k;
                two_n[i] = 2 * h->N;
                const long long len = 2LL * h->N + 3LL * h->n_b;
                B->off[i + 1] = B->off[i] + (len + 1) / 2 * 2;  // even: every system starts 16-byte aligned
                B->f_off[i + 1] = B->f_off[i] + 3LL * h->n_b;
                B->s_off[i + 1] = B->s_off[i] + 2LL * h->N;
            }
        B->n_all = B->off[n];
        B->ld = (B->n_all + 31) / 32 * 32;
        const size_t L = B->ld, mm = B->m;
        auto dalloc = [](void** p, size_t bytes) { return cudaMalloc(p, bytes) == cudaSuccess; };
        bool ok = dalloc((void**)&B->V, 8 * L * (mm + 1)) && dalloc((void**)&B->Z, 8 * L * mm) &&
                  dalloc((void**)&B->w, 8 * L) && dalloc((void**)&B->b, 8 * L) && dalloc((void**)&B->x, 8 * L) &&
                  dalloc((void**)&B->r, 8 * L) && dalloc((void**)&B->d, 8 * L) && dalloc((void**)&B->vin, 8 * L) &&
                  dalloc((void**)&B->zout, 8 * L) && dalloc((void**)&B->wout, 8 * L) &&
                  dalloc((void**)&B->dots, 8 * 3 * (size_t)n * (mm + 1)) &&
                  dalloc((void**)&B->hv, 8 * (size_t)n * (mm + 1)) &&
                  dalloc((void**)&B->d_off, sizeof(long long) * (n + 1)) &&
                  dalloc((void**)&B->d_f_off, sizeof(long long) * (n + 1)) &&
                  dalloc((void**)&B->d_s_off, sizeof(long long) * (n + 1)) &&
                  dalloc((void**)&B->d_two_n, sizeof(int) * n);
        if (!ok) {
            cudaGetLastError();
            fbim::set_global_error("fbim_batch_create: device allocation failed");
            fbim_batch_destroy(B);
            return FBIM_ERR_OOM;
        }
        const int nb = std::min(n_handles, kMaxBranches);
        B->side.resize(nb);
        B->side_ev.resize(nb);
        bool sok = cudaEventCreateWithFlags(&B->fork_ev, cudaEventDisableTiming) == cudaSuccess &&
                   cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) == cudaSuccess;
        for (int b = 0; b < nb && sok; ++b)
            sok = cudaStreamCreateWithFlags(&B->side[b], cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&B->side_ev[b], cudaEventDisableTiming) == cudaSuccess;
        // padding entries of the fixed operator buffers stay zero
        sok = sok && cudaMemsetAsync(B->vin, 0, 8 * L, B->stream) == cudaSuccess &&
              cudaMemsetAsync(B->zout, 0, 8 * L, B->stream) == cudaSuccess &&
              cudaMemsetAsync(B->wout, 0, 8 * L, B->stream) == cudaSuccess &&
              cudaMemcpyAsync(B->d_off, B->off.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice,
                              B->stream) == cudaSuccess &&
              cudaMemcpyAsync(B->d_f_off, B->f_off.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice,
                              B->stream) == cudaSuccess &&
              cudaMemcpyAsync(B->d_s_off, B->s_off.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice,
                              B->stream) == cudaSuccess &&
              cudaMemcpyAsync(B->d_two_n, two_n.data(), sizeof(int) * n, cudaMemcpyHostToDevice, B->stream) ==
                  cudaSuccess &&
              cudaStreamSynchronize(B->stream) == cudaSuccess;
        if (!sok) {
            fbim::set_global_error(std::string("fbim_batch_create: ") + cudaGetErrorString(cudaGetLastError()));
            fbim_batch_destroy(B);
            return FBIM_ERR_CUDA;
        }
        *out = B;
        return FBIM_OK;
    } catch (...) {
        fbim::set_global_error("fbim_batch_create: unexpected host exception");
        fbim_batch_destroy(B);
        return FBIM_ERR_SETUP;
    }
}

extern "C" const char* fbim_batch_last_error(fbim_batch B) { return B ? B->err.c_str() : fbim::global_error(); }

extern "C" fbim_status fbim_batch_solve(fbim_batch B, const double* F_dev, const double* slip_dev, double tol,
                                        int max_iter, double* U_dev, int* iters, double* rel_residual) {
    if (!B || !F_dev || !U_dev || !(tol > 0) || max_iter <= 0) return FBIM_ERR_INVALID_ARG;
    try {
        if (cudaSetDevice(B->device) != cudaSuccess) return FBIM_ERR_CUDA;
        return batch_solve(B, F_dev, slip_dev, tol, max_iter, U_dev, iters, rel_residual);
    } catch (...) {
        return fail(B, "unexpected host exception in fbim_batch_solve", FBIM_ERR_SETUP);
    }
}

extern "C" fbim_status fbim_batch_get_info(fbim_batch B, fbim_batch_info* info) {
    if (!B || !info) return FBIM_ERR_INVALID_ARG;
    info->n_handles = B->n_h;
    info->n_systems = B->n_tot;
    info->n_unknowns = B->n_all;
    info->restart = B->m;
    info->branches = (int)B->side.size();
    for (int k = 0; k < 4; ++k) info->graph_kernels[k] = B->g_kernels[k];
    info->launches = B->launches;
    info->graph_launches = B->graph_launches;
    return FBIM_OK;
}
