// Grid autotuner.  The grid rule of Sec. 3.2 gives the smallest FFT side M_min
// that meets the wave-space tolerance; any larger M keeps the error below it
// (finer grid, same support P and the Gaussian shape eta_s recomputed for h).
// cuFFT's speed depends strongly on the factorisation of M, so the setup times
// the forward + inverse transform pair of a few admissible sizes in
// [M_min, 1.3 M_min] (multiples of 4, 2^a 3^b 5^c 7^d, with a wave-space tile side in
// [max(16, (P - 1)/2), 64] dividing M) and keeps the cheapest.  FP32 handles
// weigh the FP64 transform (used by the refinement residuals) at 0.1 and take
// 5-smooth sides only, which their float-float FFT supports.  The smallest side
// within 5% of the cheapest is kept.
#include <cufft.h>

#include <algorithm>
#include <string>
#include <vector>

#include "fbim_internal.h"

namespace fbim {

static bool nice(int m, bool seven) {
    int r = m;
    for (int f : {2, 3, 5, 7})
        while ((f != 7 || seven) && r % f == 0) r /= f;
    return r == 1;
}

static int tile_side(int m) {
    int best = 0;
    for (int d = 1; d <= 64 && d <= m; ++d)
        if (m % d == 0) best = d;
    return best;
}

// Mean time (ms) of forward + inverse batch-2 transforms of side M, or < 0 on failure.
static double time_fft(cudaStream_t st, int M, bool fp32, void* grid, void* spec, cudaEvent_t e0, cudaEvent_t e1) {
    const int Mh = M / 2 + 1;
    int n[2] = {M, M}, inembed[2] = {M, M}, onembed[2] = {M, Mh};
    cufftHandle pf = 0, pi = 0;
    double ms = -1.0;
    if (cufftPlanMany(&pf, 2, n, inembed, 1, M * M, onembed, 1, M * Mh, fp32 ? CUFFT_R2C : CUFFT_D2Z, 2) ==
            CUFFT_SUCCESS &&
        cufftPlanMany(&pi, 2, n, onembed, 1, M * Mh, inembed, 1, M * M, fp32 ? CUFFT_C2R : CUFFT_Z2D, 2) ==
            CUFFT_SUCCESS &&
        cufftSetStream(pf, st) == CUFFT_SUCCESS && cufftSetStream(pi, st) == CUFFT_SUCCESS) {
        auto run = [&]() {
            if (fp32) {
                cufftExecR2C(pf, (float*)grid, (cufftComplex*)spec);
                cufftExecC2R(pi, (cufftComplex*)spec, (float*)grid);
            } else {
                cufftExecD2Z(pf, (double*)grid, (cufftDoubleComplex*)spec);
                cufftExecZ2D(pi, (cufftDoubleComplex*)spec, (double*)grid);
            }
        };
        run();
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3; ++r) run();
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) == cudaSuccess) {
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            ms = t / 3.0;
        }
    }
    if (pf) cufftDestroy(pf);
    if (pi) cufftDestroy(pi);
    cudaGetLastError();
    return ms;
}

fbim_status tune_grid(fbim_handle_s* h, int M_min, int P, int& M_out, double& best_ms) {
    std::vector<int> cand;
    const int ts_min = std::max(16, (P - 1) / 2);
    // multiples of 4 (the FP32 wave-space kernels then move float4 chunks)
    for (int m = (M_min + 3) / 4 * 4; m <= (int)(1.3 * M_min) + 4 && cand.size() < 12; m += 4)
        if (nice(m, h->precision != FBIM_FP32) && tile_side(m) >= ts_min) cand.push_back(m);
    M_out = M_min;
    best_ms = 0;
    if (cand.size() <= 1) {
        if (!cand.empty()) M_out = cand[0];
        return FBIM_OK;
    }
    const int Mx = cand.back();
    const size_t gbytes = 2 * (size_t)Mx * Mx * sizeof(double);
    const size_t sbytes = 2 * (size_t)Mx * (Mx / 2 + 1) * 2 * sizeof(double);
    void *grid = nullptr, *spec = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&grid, gbytes) != cudaSuccess || cudaMalloc(&spec, sbytes) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaFree(grid);
        cudaFree(spec);
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        M_out = cand[0];
        return FBIM_OK;  // tuning is optional: keep the rule's size
    }
    cudaMemsetAsync(grid, 0, gbytes, h->stream);
    const bool f32 = h->precision == FBIM_FP32;
    std::vector<double> cost(cand.size(), -1.0);
    double best = 1e300;
    for (size_t c = 0; c < cand.size(); ++c) {
        const double t = f32 ? time_fft(h->stream, cand[c], true, grid, spec, e0, e1) : 0.0;
        const double t64 = time_fft(h->stream, cand[c], false, grid, spec, e0, e1);
        if (t < 0 || t64 < 0) continue;
        cost[c] = f32 ? t + 0.1 * t64 : t64;
        best = std::min(best, cost[c]);
    }
    // the smallest side within 5% of the cheapest: timing noise does not flip the choice
    for (size_t c = 0; c < cand.size(); ++c)
        if (cost[c] >= 0 && cost[c] <= 1.05 * best) {
            M_out = cand[c];
            best_ms = cost[c];
            break;
        }
    cudaFree(grid);
    cudaFree(spec);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    return FBIM_OK;
}

}  // namespace fbim
