// Preconditioner and Krylov workspace of a handle (solver.cu, brownian.cu).
#pragma once
#include <cublas_v2.h>

#include <cmath>
#include <vector>

struct fbim_handle_s;

// Device-driven classical Gram-Schmidt state of a Krylov basis (the Lanczos iteration of
// the near-field square root; solver.cu): the index of the newest basis vector on the
// device, the step history (two passes of coefficients, |w|^2, 1/|w| per row) with its
// mapped host copy, and the block partials of the fused sweeps.
struct CgsState {
    int m = 0;                   // history rows m + 1
    int n = 0, ld = 0, nb = 0;   // vector length, basis row stride, sweep blocks
    int* kd = nullptr;
    unsigned* count = nullptr;
    double* hist = nullptr;
    double* hist_host = nullptr;
    double* hist_map = nullptr;
    double* part = nullptr;
};

// A reference block B_ref laid out for the tensor-core block operator (block_tc.cu):
// TF32 high and low parts in chunks of 32 K-columns and M-tiles of 128 rows.
struct TcBlock {
    float* A = nullptr;
    int n2 = 0, KP = 0, MT = 0, KC = 0;
    bool ready = false;  // false: 2 n_p > 256, the library GEMM serves this block
};

struct Solver {
    int n2 = 0;                 // 2 n_p
    int n = 0;                  // 2N + 3 n_b
    int ld = 0;                 // leading dimension of V and Z: n rounded up to 32 (keeps rows 16-byte aligned)
    double* Mpinv64 = nullptr;  // [n2][n2] M_ref^+
    float* Mpinv32 = nullptr;
    double* H64 = nullptr;      // [3][n2] column-major (n2 x 3): M_ref^+ K_ref
    float* H32 = nullptr;
    double Nt[9] = {};          // N~_ref, row-major
    double* G64 = nullptr;      // [n2][n2] G_ref = M(r)_ref^{-1/2} (principal, spurious modes dropped)
    double* Gd64 = nullptr;     // [n2][n2] G_ref^+ = M(r)_ref^{1/2}
    float* G32 = nullptr;
    float* Gd32 = nullptr;
    int restart = 0;
    double* V = nullptr;        // [(m+1)][ld] Krylov basis
    double* Z = nullptr;        // [m][ld] preconditioned basis
    double* w = nullptr;        // [n]
    double* r = nullptr;        // [n]
    double* d = nullptr;        // [n]
    double* t = nullptr;        // [n]
    double* hcol = nullptr;     // [m+1] the cycle's least-squares solution y (x += Z y)
    // device-driven Arnoldi step (solver.cu): index of the newest basis vector, the step
    // history (one row per step: two passes of coefficients, |w|^2, 1/|w|), its mapped
    // host mirror, and one event per step in flight
    int* kd = nullptr;
    unsigned* cg_count = nullptr;  // blocks of the running Gram-Schmidt sweep that have finished
    double* hist = nullptr;       // [(m+1)][2 (m+1) + 2]
    double* hist_host = nullptr;  // same, mapped pinned host memory, then [m+1] for y
    double* hist_map = nullptr;   // its device address
    cudaEvent_t ev_step[2] = {nullptr, nullptr};
    void* zbuf = nullptr;       // [N][2] rotated residual (T)
    void* gbuf = nullptr;       // [N][2] M_ref^+ z (T)
    cublasHandle_t blas = nullptr;
    int lanczos_max = 0;        // Lanczos workspace (brownian.cu)
    double* lz = nullptr;       // [lanczos_max][2N] Lanczos basis
    double* lh = nullptr;       // [2 lanczos_max] Lanczos dot products / coefficients
    void* blas_ws = nullptr;    // fixed cuBLAS workspace (so captured graphs never allocate)
    double* corr = nullptr;     // [n] refinement correction
    bool have_x = false;        // d holds the last solve's solution (a warm start can use it)
    // captured Arnoldi step per precision, [0] FP32 / [1] FP64: gz = P gin, gw = A gz,
    // orthogonalised and normalised into V and gin; recaptured when the handle's layout changes
    double *gin = nullptr, *gz = nullptr, *gw = nullptr;
    double* cg_part = nullptr;  // [m+1][blocks] partial dot products of the fused Gram-Schmidt
    cudaGraphExec_t op_graph[2] = {nullptr, nullptr};
    unsigned long long op_version[2] = {0, 0};
    long long op_kernels[2] = {0, 0};
    cudaStream_t cap = nullptr;  // capture origin (the handle's stream may be the legacy default)
    double* rfd = nullptr;      // [2N + 6 * 3 n_b] workspace of the random-finite-difference step
    // FP32 handles: |(A_32 - A_64) v| / |v| for a random v, measured on the first solve; it
    // bounds the error of a residual advanced with the FP32 operator (r - A_32 d)
    double e32 = -1.0;
    // tensor-core block operators of FBIM_FP32 handles: M_ref^+ (preconditioner), G_ref and
    // G_ref^+ (near-field square root); tc_err = device flag of a timed-out wait
    TcBlock tc_Mp, tc_G, tc_Gd;
    int* tc_err = nullptr;
    // dot products: block partials, finished-block count, and the result's mapped host slot
    double* dot_part = nullptr;
    unsigned* dot_count = nullptr;
    double* dot_host = nullptr;
    double* dot_map = nullptr;
    // Lanczos (brownian.cu): Gram-Schmidt state over the basis lz, the step input, the
    // orthogonalised vector and the coefficients of the final combination
    CgsState lan;
    double* lan_in = nullptr;
    double* lan_w = nullptr;
    double* lan_c = nullptr;
};

namespace fbim {
fbim_status tc_prepare(fbim_handle_s* h, const std::vector<double>& Bref, int n2, TcBlock& out);
void tc_free(TcBlock& b);
// mode 0: out_b = R_b B_ref R_b^T in_b; 1: out_g = B_ref R_b^T in_b (FP32, body frame);
// 2: the preconditioner's body solve (out = mu, out_U = U) with H and N~ (row-major)
fbim_status tc_apply(fbim_handle_s* h, const TcBlock& B, int mode, const double* in, double* out, double* out_U,
                     float* out_g, const float* H, const double* Nt, int* err);
// FBIM_ERR_TIMEOUT when a tensor-core block kernel gave up a wait (host-synchronising)
fbim_status tc_check(fbim_handle_s* h);
// vector kernels of the solvers (solver.cu): <x, y> and |x| (host-synchronising), and
// y = beta y + sum_{j < k} c_j V_j with c on the device
fbim_status dev_dot(fbim_handle_s* h, int n, const double* x, const double* y, double& out);
fbim_status dev_norm2(fbim_handle_s* h, int n, const double* x, double& out);
void dev_combine(fbim_handle_s* h, int n, int k, const double* V, int ld, const double* c, double beta, double* y);
fbim_status cgs_alloc(fbim_handle_s* h, CgsState& c, int n, int ld, int m);
void cgs_free(CgsState& c);
int cgs_hist_stride(int m);
void cgs_start(fbim_handle_s* h, CgsState& c, double a, const double* w, double* V, double* next_in);
void cgs_step(fbim_handle_s* h, CgsState& c, double* V, double* w, bool two_pass, double* next_in);
}  // namespace fbim
