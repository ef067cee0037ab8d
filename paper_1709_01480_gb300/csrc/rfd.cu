// Brownian dynamics steps with a random finite difference (Sec. 4.4).
//
// Euler-Maruyama (Eq. EM-RFD):
//   Q^{n+1} = Q^n + dt N F + sqrt(2 kT dt) N^1/2 W
//             + dt kT/delta [ N(Q + delta/2 W~) W~ - N(Q - delta/2 W~) W~ ].
// The first two terms are dt U with U from one saddle solve with right-hand side
// [slip; F], slip = sqrt(2kT/dt) M^1/2 W (fbim_brownian_slip); the drift needs two
// solves with force W~ and no slip at the displaced configurations.  Three solves
// per step, as in the paper.  W~ is drawn from Philox stream 2 (or given).
//
// Adams-Bashforth (Eq. AB2-RFD): the deterministic part becomes
// dt (3/2 N^n F^n - 1/2 N^{n-1} F^{n-1}), so N^n F^n is solved apart from the slip's
// velocity (force zero): four solves per step; N F is carried to the next step.
//
// Either scheme may solve the RFD pair at a looser tolerance than the rest (Sec. 4.4.2
// solves them at 1e-3 with the deterministic solves at 1e-6).
#include <cmath>

#include "ewald_types.cuh"
#include "fbim_internal.h"
#include "solver.cuh"

namespace fbim {

fbim_status mobility_solve(fbim_handle_s* h, const double* F, const double* slip, double tol, int max_iter,
                           double* U, double* mu_out, int* iters_out, double* res_out, bool warm);
fbim_status brownian_slip(fbim_handle_s* h, unsigned long long seed, unsigned long long counter, double kT, double dt,
                          const double* W_r, const double* Z_w, double tol, int max_iter, double* slip,
                          int* lanczos_iters);

fbim_status ensure_solver(fbim_handle_s* h);

namespace {

__global__ void k_wtilde(int n, unsigned long long seed, unsigned counter, double* __restrict__ w) {
    int blk = blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * blk >= n) return;
    double2 z = philox_normals(seed, 2u, counter, (unsigned long long)blk);
    w[2 * blk] = z.x;
    if (2 * blk + 1 < n) w[2 * blk + 1] = z.y;
}

__global__ void k_displace(int n, const double* __restrict__ Q, double a, const double* __restrict__ w,
                           double* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = Q[i] + a * w[i];
}

// Up, Um null: Q += dt U (no random finite difference)
__global__ void k_rfd_update(long long n, double* __restrict__ Q, double dt, const double* __restrict__ U, double c,
                             const double* __restrict__ Up, const double* __restrict__ Um) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Q[i] += Up ? dt * U[i] + c * (Up[i] - Um[i]) : dt * U[i];
}

// Q += dt (U_noise + 3/2 Ud - 1/2 NF_prev) + c (Up - Um); NF_prev NULL: dt (U_noise + Ud)
__global__ void k_ab2_update(int n, double* __restrict__ Q, double dt, const double* __restrict__ Un,
                             const double* __restrict__ Ud, const double* __restrict__ NFp, double c,
                             const double* __restrict__ Up, const double* __restrict__ Um) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double det = NFp ? 1.5 * Ud[i] - 0.5 * NFp[i] : Ud[i];
    Q[i] += dt * (Un[i] + det) + c * (Up[i] - Um[i]);
}

}  // namespace

fbim_status bd_step(fbim_handle_s* h, int scheme, const double* F, double dt, double kT, double delta,
                    unsigned long long seed, unsigned long long step, const double* W_r, const double* Z_w,
                    const double* W_t, double tol, double tol_rfd, int max_iter, double* NF, int have_prev, double* Q,
                    int* iters_total) {
    const int n3 = 3 * h->n_b, n2 = 2 * h->N, tb = 256;
    const bool ab2 = scheme == FBIM_AB2;
    const bool no_rfd = scheme == FBIM_EM_NO_RFD;
    // work: slip [2N], W~, Q+-, U, U+, U-, U_det, zero [3 n_b each] (kept in the solver workspace)
    FBIM_TRY(ensure_solver(h));
    Solver* S = h->solver;
    if (!S->rfd) FBIM_CUDA_TRY(h, cudaMalloc(&S->rfd, sizeof(double) * (n2 + 8 * (size_t)n3)));
    double* work = S->rfd;
    double* slip = work;
    double* wt = slip + n2;
    double* Qd = wt + n3;
    double* U = Qd + n3;
    double* Up = U + n3;
    double* Um = Up + n3;
    double* Ud = Um + n3;
    double* zero = Ud + n3;
    fbim_status st = FBIM_OK;
    int it = 0, total = 0;
    auto run = [&]() -> fbim_status {
        // (1) geometry at Q (already in place when the previous step left the handle
        // there), slip, and the velocity: EM N F + N^1/2 W in one solve; AB2 the slip's
        // velocity (force zero) and N F apart
        FBIM_TRY(update_positions_if_moved(h, Q));
        int lz = 0;
        FBIM_TRY(brownian_slip(h, seed, 3 * step, kT, dt, W_r, Z_w, std::max(tol, 1e-12), 200, slip, &lz));
        fbim_status s0 = FBIM_OK;
        if (ab2) FBIM_CUDA_TRY(h, cudaMemsetAsync(zero, 0, sizeof(double) * n3, h->stream));
        fbim_status s1 = mobility_solve(h, ab2 ? zero : F, slip, tol, max_iter, U, nullptr, &it, nullptr, false);
        total += it;
        if (s1 != FBIM_OK && s1 != FBIM_ERR_NOT_CONVERGED) return s1;
        if (ab2) {
            s0 = mobility_solve(h, F, nullptr, tol, max_iter, Ud, nullptr, &it, nullptr, false);
            total += it;
            if (s0 != FBIM_OK && s0 != FBIM_ERR_NOT_CONVERGED) return s0;
        }
        if (no_rfd) {  // Eq. EM-noRFD: Q += dt (N F + N^1/2 W), no stochastic drift
            k_rfd_update<<<(n3 + tb - 1) / tb, tb, 0, h->stream>>>(n3, Q, dt, U, 0.0, nullptr, nullptr);
            h->launches += 1;
            FBIM_CUDA_TRY(h, cudaGetLastError());
            FBIM_TRY(update_positions(h, Q));
            return s1 != FBIM_OK ? FBIM_ERR_NOT_CONVERGED : FBIM_OK;
        }
        // (2) random finite difference of N along W~
        if (W_t) {
            FBIM_CUDA_TRY(h, cudaMemcpyAsync(wt, W_t, sizeof(double) * n3, cudaMemcpyDeviceToDevice, h->stream));
        } else {
            k_wtilde<<<(n3 / 2 + tb) / tb, tb, 0, h->stream>>>(n3, seed, (unsigned)step, wt);
        }
        k_displace<<<(n3 + tb - 1) / tb, tb, 0, h->stream>>>(n3, Q, 0.5 * delta, wt, Qd);
        FBIM_TRY(update_positions(h, Qd));
        fbim_status s2 = mobility_solve(h, wt, nullptr, tol_rfd, max_iter, Up, nullptr, &it, nullptr, false);
        total += it;
        if (s2 != FBIM_OK && s2 != FBIM_ERR_NOT_CONVERGED) return s2;
        k_displace<<<(n3 + tb - 1) / tb, tb, 0, h->stream>>>(n3, Q, -0.5 * delta, wt, Qd);
        FBIM_TRY(update_positions(h, Qd));
        // same force at a configuration 2 delta/2 |W~| away: start from the Q+ solution
        fbim_status s3 = mobility_solve(h, wt, nullptr, tol_rfd, max_iter, Um, nullptr, &it, nullptr, true);
        total += it;
        if (s3 != FBIM_OK && s3 != FBIM_ERR_NOT_CONVERGED) return s3;
        // (3) update and leave the handle at the new configuration
        if (ab2) {
            k_ab2_update<<<(n3 + tb - 1) / tb, tb, 0, h->stream>>>(n3, Q, dt, U, Ud, have_prev ? NF : nullptr,
                                                                   dt * kT / delta, Up, Um);
            FBIM_CUDA_TRY(h, cudaMemcpyAsync(NF, Ud, sizeof(double) * n3, cudaMemcpyDeviceToDevice, h->stream));
        } else {
            k_rfd_update<<<(n3 + tb - 1) / tb, tb, 0, h->stream>>>(n3, Q, dt, U, dt * kT / delta, Up, Um);
        }
        h->launches += (W_t ? 0 : 1) + 3;
        FBIM_CUDA_TRY(h, cudaGetLastError());
        FBIM_TRY(update_positions(h, Q));
        if (s0 != FBIM_OK || s1 != FBIM_OK || s2 != FBIM_OK || s3 != FBIM_OK) return FBIM_ERR_NOT_CONVERGED;
        return FBIM_OK;
    };
    st = run();
    cudaStreamSynchronize(h->stream);
    if (iters_total) *iters_total = total;
    return st;
}

fbim_status rfd_step(fbim_handle_s* h, const double* F, double dt, double kT, double delta, unsigned long long seed,
                     unsigned long long step, const double* W_r, const double* Z_w, const double* W_t, double tol,
                     int max_iter, double* Q, int* iters_total) {
    return bd_step(h, FBIM_EM, F, dt, kT, delta, seed, step, W_r, Z_w, W_t, tol, tol, max_iter, nullptr, 0, Q,
                   iters_total);
}

}  // namespace fbim

extern "C" fbim_status fbim_bd_step(fbim_handle h, int scheme, const double* F_dev, double dt, double kT,
                                    double delta, uint64_t seed, uint64_t step, const double* W_r_dev,
                                    const double* Z_w_dev, const double* W_t_dev, double tol, double tol_rfd,
                                    int max_iter, double* NF_dev, int have_prev, double* Q_dev, int* iters) {
    if (!h || !F_dev || !Q_dev || !(dt > 0) || !(kT >= 0) || !(delta > 0) || !(tol > 0) || !(tol_rfd > 0) ||
        max_iter <= 0 || (scheme != FBIM_EM && scheme != FBIM_AB2 && scheme != FBIM_EM_NO_RFD) ||
        (scheme == FBIM_AB2 && !NF_dev))
        return FBIM_ERR_INVALID_ARG;
    try {
        if (cudaSetDevice(h->device) != cudaSuccess) return FBIM_ERR_CUDA;
        return fbim::bd_step(h, scheme, F_dev, dt, kT, delta, seed, step, W_r_dev, Z_w_dev, W_t_dev, tol, tol_rfd,
                             max_iter, NF_dev, have_prev, Q_dev, iters);
    } catch (...) {
        h->fail("unexpected host exception in fbim_bd_step");
        return FBIM_ERR_SETUP;
    }
}

extern "C" fbim_status fbim_rfd_step(fbim_handle h, const double* F_dev, double dt, double kT, double delta,
                                     uint64_t seed, uint64_t step, const double* W_r_dev, const double* Z_w_dev,
                                     const double* W_t_dev, double tol, int max_iter, double* Q_dev, int* iters) {
    if (!h || !F_dev || !Q_dev || !(dt > 0) || !(kT >= 0) || !(delta > 0) || !(tol > 0) || max_iter <= 0)
        return FBIM_ERR_INVALID_ARG;
    try {
        if (cudaSetDevice(h->device) != cudaSuccess) return FBIM_ERR_CUDA;
        return fbim::rfd_step(h, F_dev, dt, kT, delta, seed, step, W_r_dev, Z_w_dev, W_t_dev, tol, max_iter, Q_dev,
                              iters);
    } catch (...) {
        h->fail("unexpected host exception in fbim_rfd_step");
        return FBIM_ERR_SETUP;
    }
}

extern "C" fbim_status fbim_bd_update(void* stream, size_t n, double dt, double c, const double* U_dev,
                                      const double* Up_dev, const double* Um_dev, double* Q_dev) {
    if (!U_dev || !Q_dev || (!Up_dev) != (!Um_dev) || !std::isfinite(dt) || !std::isfinite(c) ||
        n > (size_t)1 << 38)
        return FBIM_ERR_INVALID_ARG;
    if (n == 0) return FBIM_OK;
    const int tb = 256;
    fbim::k_rfd_update<<<(unsigned)((n + tb - 1) / tb), tb, 0, (cudaStream_t)stream>>>(
        (long long)n, Q_dev, dt, U_dev, c, Up_dev, Um_dev);
    return cudaGetLastError() == cudaSuccess ? FBIM_OK : FBIM_ERR_CUDA;
}
