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
//
// Batched Brownian slip (Sec. 3.3, Eq. sqrtM-split; Sec. 3.4, Eq. Gprecond-decomp):
// the near field of every system by one Lanczos iteration over the stacked vector
// (a graph of G M(r) G^T per step, segmented classical Gram-Schmidt twice in FP64,
// segment norms and normalisation on the device, the next step queued before the
// host reads the last one's alpha and beta), each system stopping on its own test;
// then a graph of G^+ and each system's far-field noise on the branch streams.  The
// iteration starts, as the single slip's does, from G^+ G W(r), W(r)'s projection onto
// the range of G.
#include <cublas_v2.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "ewald_types.cuh"
#include "fbim_internal.h"
#include "lanczos_host.h"
#include "solver.cuh"

constexpr int kGraphs = 7;

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
    // graphs: [0] precondition + saddle FP32, [1] same FP64, [2] saddle FP32, [3] saddle FP64,
    // [4] G M(r) G^T, [5] G^+ and [6] G^+ G in the handles' precision (the Brownian slip)
    cudaGraphExec_t g[kGraphs] = {};
    long long g_kernels[kGraphs] = {};       // this library's kernels in each graph
    std::vector<unsigned long long> g_version[kGraphs];
    // batched Lanczos workspace (grown on demand)
    int lz_cap = 0;                          // basis vectors held
    double* lz_V = nullptr;                  // [lz_cap][ld] basis V_0, V_1, ...
    double* lz_dots = nullptr;               // [3][n_tot][lz_cap] the two Gram-Schmidt passes, the norm
    double* lz_coef = nullptr;               // [n_tot][lz_cap] coefficients of the final combination
    int* lz_cnt = nullptr;                   // [n_tot] basis vectors each combination uses
    int* lz_active = nullptr;                // [n_tot] 1 while the system's iteration runs
    double* lz_rec = nullptr;                // mapped host [lz_cap][n_tot][2]: alpha_k, |w_k|^2
    double* lz_rec_dev = nullptr;            // its device address
    unsigned long long* d_seeds = nullptr;   // [n_tot]
    cudaEvent_t lz_ev[2] = {nullptr, nullptr};
    std::vector<int> lz_active_host;
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

// Near-field normals W(r) of every system into the stacked vector (zero past 2N):
// the Philox draws of fbim_brownian_slip with the system's seed (stream 0; FP32
// transform for FP32 handles).  One thread per pair: segments start even and 2N
// is even, so a pair never straddles two systems.
__global__ void k_batch_normals(long long n_pairs, const long long* __restrict__ off, int n_seg,
                                const int* __restrict__ two_n, const unsigned long long* __restrict__ seeds,
                                unsigned counter, int f32, double* __restrict__ out) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs) return;
    const long long t = 2 * p;
    const int i = seg_of(off, n_seg, t);
    const long long k = t - off[i];
    double2 z = make_double2(0.0, 0.0);
    if (k < two_n[i]) {
        if (f32) {
            const float2 zf = fbim::philox_normals_f(seeds[i], 0u, counter, (unsigned long long)(k / 2));
            z = make_double2(zf.x, zf.y);
        } else {
            z = fbim::philox_normals(seeds[i], 0u, counter, (unsigned long long)(k / 2));
        }
    }
    out[t] = z.x;
    out[t + 1] = z.y;
}

// V_next = w / |w| per system while it is active (|w|^2 = nrm[i * stride]); exact zeros
// for a stopped system, so that nothing it leaves behind reaches later steps
__global__ void k_seg_normalize(long long n_all, const long long* __restrict__ off, int n_seg,
                                const double* __restrict__ nrm, int stride, const int* __restrict__ active,
                                const double* __restrict__ w, double* __restrict__ v_next) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_all) return;
    const int i = seg_of(off, n_seg, t);
    const double q = nrm[(size_t)i * stride];
    const bool on = active[i] != 0 && q > 0.0 && isfinite(q);
    v_next[t] = on ? w[t] * rsqrt(q) : 0.0;
}

// alpha_k = <v_k, A v_k> (the k-th coefficients of the two Gram-Schmidt passes) and
// |w_k|^2 of every system into row k of the mapped host record
__global__ void k_lz_record(int n_seg, int k, int stride, const double* __restrict__ d1,
                            const double* __restrict__ d2, const double* __restrict__ nrm, double* __restrict__ rec) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_seg) return;
    rec[2 * i] = d1[(size_t)i * stride + k] + d2[(size_t)i * stride + k];
    rec[2 * i + 1] = nrm[(size_t)i * stride];
}

// out = sum_{j < cnt[i]} a[i][j] V_j on system i's segment (terms past a system's own
// count are never read)
__global__ void k_seg_combine_cnt(long long n_all, const long long* __restrict__ off, int n_seg,
                                  const int* __restrict__ cnt, const double* __restrict__ a, int stride,
                                  const double* __restrict__ V, long long ld, double* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_all) return;
    const int i = seg_of(off, n_seg, t);
    double v = 0.0;
    for (int j = 0; j < cnt[i]; ++j) v += a[(size_t)i * stride + j] * V[(size_t)j * ld + t];
    out[t] = v;
}

// slip = sc (near + far) into the caller's stacked [2N] blocks
__global__ void k_batch_slip_out(long long n_all, const long long* __restrict__ off, int n_seg,
                                 const int* __restrict__ two_n, const long long* __restrict__ s_off, double sc,
                                 const double* __restrict__ near, const double* __restrict__ far,
                                 double* __restrict__ slip) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_all) return;
    const int i = seg_of(off, n_seg, t);
    const long long k = t - off[i];
    if (k < two_n[i]) slip[s_off[i] + k] = sc * (near[t] + far[t]);
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
// (FP32 / FP64 operator), kind 2/3 = saddle only (FP32 / FP64), kind 4 = G M(r) G^T
// and kind 6 = G^+ G on the first 2N entries (the rest of the segment set to zero),
// kind 5 = G^+.
fbim_status system_ops(fbim_batch B, int i, int kind) {
    fbim_handle h = B->hs[B->h_of[i]];
    const bool fp32 = (kind & 1) == 0;
    const double* in = B->vin + B->off[i];
    double* z = B->zout + B->off[i];
    double* y = B->wout + B->off[i];
    if (kind == 4 || kind == 6) {
        BSTATUS(kind == 4 ? fbim::lanczos_operator(h, in, y) : fbim::g_project(h, in, y));
        const long long tail = B->off[i + 1] - B->off[i] - 2LL * h->N;
        BTRY(cudaMemsetAsync(y + 2LL * h->N, 0, sizeof(double) * tail, h->stream));
        return FBIM_OK;
    }
    if (kind == 5) return fbim::gplus_apply(h, in, y);
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

// Batched Lanczos workspace for up to cap basis vectors (grown on demand).
fbim_status ensure_lanczos(fbim_batch B, int cap) {
    if (B->lz_cap >= cap) return FBIM_OK;
    cudaFree(B->lz_V);
    cudaFree(B->lz_dots);
    cudaFree(B->lz_coef);
    if (B->lz_rec) cudaFreeHost(B->lz_rec);
    B->lz_V = B->lz_dots = B->lz_coef = B->lz_rec = B->lz_rec_dev = nullptr;
    B->lz_cap = 0;
    const size_t n = B->n_tot;
    BTRY(cudaMalloc(&B->lz_V, sizeof(double) * (size_t)B->ld * cap));
    BTRY(cudaMalloc(&B->lz_dots, sizeof(double) * 3 * n * cap));
    BTRY(cudaMalloc(&B->lz_coef, sizeof(double) * n * cap));
    BTRY(cudaHostAlloc(&B->lz_rec, sizeof(double) * 2 * n * cap, cudaHostAllocMapped));
    BTRY(cudaHostGetDevicePointer(&B->lz_rec_dev, B->lz_rec, 0));
    if (!B->lz_cnt) {
        BTRY(cudaMalloc(&B->lz_cnt, sizeof(int) * n));
        BTRY(cudaMalloc(&B->lz_active, sizeof(int) * n));
        BTRY(cudaMalloc(&B->d_seeds, sizeof(unsigned long long) * n));
        BTRY(cudaEventCreateWithFlags(&B->lz_ev[0], cudaEventDisableTiming));
        BTRY(cudaEventCreateWithFlags(&B->lz_ev[1], cudaEventDisableTiming));
    }
    B->lz_cap = cap;
    return FBIM_OK;
}

template <typename T>
fbim_status far_fields(fbim_batch B, const unsigned long long* seeds, unsigned counter, double* far) {
    // each system's (M(w))^1/2 W(w) on its handle's branch; the systems of one handle
    // share its wave-space buffers and run in turn
    const int nb = (int)B->side.size();
    BTRY(cudaEventRecord(B->fork_ev, B->stream));
    for (int b = 0; b < nb; ++b) BTRY(cudaStreamWaitEvent(B->side[b], B->fork_ev, 0));
    fbim_status st = FBIM_OK;
    for (int i = 0; i < B->n_tot && st == FBIM_OK; ++i) {
        const int k = B->h_of[i];
        fbim_handle h = B->hs[k];
        fbim::bind_stream(h, B->side[k % nb]);
        const long long l0 = h->launches;
        st = fbim::apply_noise<T>(h, nullptr, seeds[i], counter, far + B->off[i]);
        B->launches += h->launches - l0;
        if (st != FBIM_OK) B->err = std::string("batch far field: ") + h->err;
    }
    for (fbim_handle h : B->hs) fbim::bind_stream(h, B->stream);
    for (int b = 0; b < nb; ++b) {
        BTRY(cudaEventRecord(B->side_ev[b], B->side[b]));
        BTRY(cudaStreamWaitEvent(B->stream, B->side_ev[b], 0));
    }
    return st;
}

// Brownian slip of every system (see the file comment); system i's slip is that of
// fbim_brownian_slip on its handle with seed seeds[i] and the same counter.
fbim_status batch_slip(fbim_batch B, const unsigned long long* seeds, unsigned long long counter, double kT, double dt,
                       double tol, int max_iter, double* slip, int* iters_out) {
    const int n = B->n_tot, tb = 256;
    const long long N = B->n_all, ld = B->ld;
    cudaStream_t st = B->stream;
    const bool fp32 = B->hs[0]->precision == FBIM_FP32;
    const int cap = max_iter + 2;  // V_0 .. V_{max_iter + 1}: a step queued past the last one writes one more
    const int stride = cap;
    BSTATUS(ensure_lanczos(B, cap));
    BSTATUS(capture(B, 4));
    BSTATUS(capture(B, 5));
    BSTATUS(capture(B, 6));
    B->lz_active_host.assign(n, 0);
    BTRY(cudaMemcpyAsync(B->d_seeds, seeds, sizeof(unsigned long long) * n, cudaMemcpyHostToDevice, st));
    k_batch_normals<<<blocks(N / 2, tb), tb, 0, st>>>(N / 2, B->d_off, n, B->d_two_n, B->d_seeds,
                                                      (unsigned)counter, fp32 ? 1 : 0, B->x);
    B->launches += 1;
    // start from G^+ G W(r), as the single slip does: the null space of G contributes f(0) = 0
    BSTATUS(run_graph(B, 6, B->x, nullptr, B->b));
    std::vector<double> wn2, wn(n), inv(n);
    BSTATUS(seg_norms2(B, B->b, wn2));
    for (int i = 0; i < n; ++i) {
        wn[i] = std::sqrt(wn2[i]);
        inv[i] = wn[i] > 0 ? 1.0 / wn[i] : 0.0;
        B->lz_active_host[i] = wn[i] > 0 ? 1 : 0;
    }
    BSTATUS(seg_scale(B, inv, B->b, B->lz_V));  // V_0 = W / |W|
    BTRY(cudaMemcpyAsync(B->lz_active, B->lz_active_host.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    double* d1 = B->lz_dots;
    double* d2 = d1 + (size_t)n * stride;
    double* nr = d2 + (size_t)n * stride;
    // one step for every system: w = G M(r) G^T v_k, two Gram-Schmidt passes against
    // V_0..V_k, |w|^2, V_{k+1} = w / |w| while active, alpha_k and |w|^2 to the host record
    auto enqueue = [&](int k) -> fbim_status {
        BSTATUS(run_graph(B, 4, B->lz_V + (size_t)k * ld, nullptr, B->w));
        for (double* dst : {d1, d2}) {
            k_seg_dots<<<dim3(n, k + 1), 256, 0, st>>>(B->d_off, B->lz_V, ld, B->w, dst, stride);
            k_seg_update<<<blocks(N, tb), tb, 0, st>>>(N, B->d_off, n, k + 1, B->lz_V, ld, dst, stride, B->w);
        }
        k_seg_dots<<<dim3(n, 1), 256, 0, st>>>(B->d_off, B->w, 0, B->w, nr, stride);
        k_seg_normalize<<<blocks(N, tb), tb, 0, st>>>(N, B->d_off, n, nr, stride, B->lz_active, B->w,
                                                      B->lz_V + (size_t)(k + 1) * ld);
        k_lz_record<<<(n + 127) / 128, 128, 0, st>>>(n, k, stride, d1, d2, nr, B->lz_rec_dev + (size_t)2 * n * k);
        B->launches += 7;
        BTRY(cudaGetLastError());
        BTRY(cudaEventRecord(B->lz_ev[k & 1], st));
        return FBIM_OK;
    };
    std::vector<std::vector<double>> alpha(n), beta(n), coef(n);
    std::vector<double> d_last(n, -1.0), d_prev(n, -1.0);
    std::vector<int> its(n, 0);
    int n_active = 0;
    for (int i = 0; i < n; ++i) n_active += B->lz_active_host[i];
    if (n_active > 0) BSTATUS(enqueue(0));
    for (int k = 0; k < max_iter && n_active > 0; ++k) {
        // queue the next step unless every running system is predicted to stop here
        bool ahead = false;
        if (k + 1 < max_iter)
            for (int i = 0; i < n && !ahead; ++i) {
                if (!B->lz_active_host[i]) continue;
                ahead = !(d_last[i] >= 0.0 && d_prev[i] > 0.0) ||
                        d_last[i] * std::min(d_last[i] / d_prev[i], 1.0) > tol;
            }
        if (ahead) BSTATUS(enqueue(k + 1));
        BTRY(cudaEventSynchronize(B->lz_ev[k & 1]));
        const double* row = B->lz_rec + (size_t)2 * n * k;
        bool changed = false;
        for (int i = 0; i < n; ++i) {
            if (!B->lz_active_host[i]) continue;
            const double bn = std::sqrt(std::max(row[2 * i + 1], 0.0));
            alpha[i].push_back(row[2 * i]);
            beta[i].push_back(bn);
            ++its[i];
            std::vector<double> c = fbim::lanczos_sqrt_coeffs(alpha[i].data(), beta[i].data(), k + 1, wn[i]);
            double dn = 0, cn = 0;
            for (int j = 0; j <= k; ++j) {
                const double prev = j < (int)coef[i].size() ? coef[i][j] : 0.0;
                dn += (c[j] - prev) * (c[j] - prev);
                cn += c[j] * c[j];
            }
            coef[i].swap(c);
            if (!std::isfinite(bn) || !std::isfinite(cn))
                return fail(B, "batched Lanczos iterate is not finite", FBIM_ERR_NONFINITE);
            d_prev[i] = d_last[i];
            d_last[i] = cn > 0.0 ? std::sqrt(dn / cn) : 0.0;
            const bool conv = (k > 0 && std::sqrt(dn) <= tol * std::sqrt(cn)) || bn <= 1e-14 * wn[i];
            if (conv || k + 1 == max_iter) {
                B->lz_active_host[i] = 0;
                --n_active;
                changed = true;
            }
        }
        if (n_active == 0) break;
        // stop the finished systems from the next queued step on (ordered after the queued one)
        if (changed)
            BTRY(cudaMemcpyAsync(B->lz_active, B->lz_active_host.data(), sizeof(int) * n, cudaMemcpyHostToDevice,
                                 st));
        if (!ahead) BSTATUS(enqueue(k + 1));
    }
    // near = G^+ V c per system, far = its wave-space noise, slip = sqrt(2 kT / dt) (near + far)
    std::vector<double> cm((size_t)n * stride, 0.0);
    std::vector<int> cnt(n);
    for (int i = 0; i < n; ++i) {
        cnt[i] = (int)coef[i].size();
        std::copy(coef[i].begin(), coef[i].end(), cm.begin() + (size_t)i * stride);
    }
    BTRY(cudaMemcpyAsync(B->lz_coef, cm.data(), sizeof(double) * cm.size(), cudaMemcpyHostToDevice, st));
    BTRY(cudaMemcpyAsync(B->lz_cnt, cnt.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    k_seg_combine_cnt<<<blocks(N, tb), tb, 0, st>>>(N, B->d_off, n, B->lz_cnt, B->lz_coef, stride, B->lz_V, ld, B->d);
    B->launches += 1;
    BSTATUS(run_graph(B, 5, B->d, nullptr, B->r));
    if (fp32)
        BSTATUS(far_fields<float>(B, seeds, (unsigned)counter, B->x));
    else
        BSTATUS(far_fields<double>(B, seeds, (unsigned)counter, B->x));
    k_batch_slip_out<<<blocks(N, tb), tb, 0, st>>>(N, B->d_off, n, B->d_two_n, B->d_s_off, std::sqrt(2.0 * kT / dt),
                                                   B->r, B->x, slip);
    B->launches += 1;
    BTRY(cudaGetLastError());
    BTRY(cudaStreamSynchronize(st));  // the host vectors above outlive their copies
    for (fbim_handle h : B->hs) {
        const fbim_status ts = fbim::tc_check(h);
        if (ts != FBIM_OK) return fail(B, "batched slip: " + h->err, ts);
    }
    if (iters_out)
        for (int i = 0; i < n; ++i) iters_out[i] = its[i];
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
    for (double* p : {B->lz_V, B->lz_dots, B->lz_coef}) cudaFree(p);
    cudaFree(B->lz_cnt);
    cudaFree(B->lz_active);
    cudaFree(B->d_seeds);
    if (B->lz_rec) cudaFreeHost(B->lz_rec);
    for (cudaEvent_t e : B->lz_ev)
        if (e) cudaEventDestroy(e);
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
    for (int k = 0; k < kGraphs; ++k) info->graph_kernels[k] = B->g_kernels[k];
    info->launches = B->launches;
    info->graph_launches = B->graph_launches;
    return FBIM_OK;
}

extern "C" fbim_status fbim_batch_slip(fbim_batch B, const uint64_t* seeds, uint64_t counter, double kT, double dt,
                                       double tol, int max_iter, double* slip_dev, int* lanczos_iters) {
    if (!B || !seeds || !slip_dev || !(dt > 0) || !(kT >= 0) || !(tol > 0) || max_iter <= 0 || max_iter > 1000)
        return FBIM_ERR_INVALID_ARG;
    try {
        if (cudaSetDevice(B->device) != cudaSuccess) return FBIM_ERR_CUDA;
        std::vector<unsigned long long> sd(seeds, seeds + B->n_tot);
        return batch_slip(B, sd.data(), counter, kT, dt, tol, max_iter, slip_dev, lanczos_iters);
    } catch (...) {
        return fail(B, "unexpected host exception in fbim_batch_slip", FBIM_ERR_SETUP);
    }
}
