// C ABI entry points: handle life cycle and the Ewald operators.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "fbim_internal.h"

using fbim::set_global_error;

namespace {

template <typename F>
fbim_status guarded(fbim_handle h, F&& f) {
    try {
        return f();
    } catch (const std::bad_alloc&) {
        if (h) h->fail("host allocation failed");
        return FBIM_ERR_OOM;
    } catch (...) {
        if (h) h->fail("unexpected host exception");
        return FBIM_ERR_SETUP;
    }
}

void release(fbim_handle h) {
    if (!h) return;
    cudaSetDevice(h->device);
    for (auto& e : h->ev)
        if (e) cudaEventDestroy(e);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->aux) cudaStreamDestroy(h->aux);
    fbim::free_ewald(h);
    fbim::free_coarse(h);
    cudaFree(h->ref);
    cudaFree(h->Q);
    cudaFree(h->x);
    cudaFree(h->cell);
    cudaFree(h->cell_start);
    cudaFree(h->cell_fill);
    cudaFree(h->perm);
    cudaFree(h->slot);
    cudaFree(h->flags);
    cudaFree(h->band_dev);
    cudaFree(h->gbase);
    cudaFree(h->tile_start);
    cudaFree(h->tile_fill);
    cudaFree(h->tperm);
    cudaFree(h->tslot);
    cudaFree(h->tile_tmp);
    cudaFree(h->rot);
    fbim::free_second_kind(h);
    fbim::free_solver(h);
    delete h;
}

fbim_status check_flags(fbim_handle h) {
    int f[4];
    FBIM_CUDA_TRY(h, cudaMemcpyAsync(f, h->flags, sizeof(f), cudaMemcpyDeviceToHost, h->stream));
    FBIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (f[0]) {
        h->fail("non-finite body coordinates");
        return FBIM_ERR_NONFINITE;
    }
    if (f[1]) {
        h->fail("two nodes coincide (overlapping bodies)");
        return FBIM_ERR_OVERLAP;
    }
    return FBIM_OK;
}

}  // namespace

extern "C" fbim_status fbim_default_params(fbim_params* p) {
    if (!p) return FBIM_ERR_INVALID_ARG;
    std::memset(p, 0, sizeof(*p));
    p->precision = FBIM_FP64;
    p->alpert_order = 4;
    p->grid = 0;
    p->support = 0;
    p->eta = 1.0;
    p->stream = nullptr;
    p->device = 0;
    p->restart = 60;
    p->autotune = 1;
    p->grid_tune = 1;
    p->split_tune = 0;
    p->fp32_support = 0;
    p->tensor_cores = 1;
    return FBIM_OK;
}

static fbim_status setup_one(fbim_handle* out, int n_b, int n_p, const double* ref_nodes_host,
                             const double* Q_host, double L, double r_c, double xi, double tol,
                             const fbim_params* opt) {
    if (!out || n_b <= 0 || n_p < 8 || !ref_nodes_host || !Q_host || !(L > 0) || !(tol > 0 && tol < 1)) {
        set_global_error("fbim_setup: invalid argument");
        return FBIM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    fbim_params p;
    fbim_default_params(&p);
    if (opt) p = *opt;
    if (p.precision != FBIM_FP64 && p.precision != FBIM_FP32) {
        set_global_error("fbim_setup: precision must be FBIM_FP64 or FBIM_FP32");
        return FBIM_ERR_INVALID_ARG;
    }
    if ((long long)n_b * n_p > (1LL << 30)) {
        set_global_error("fbim_setup: too many nodes");
        return FBIM_ERR_INVALID_ARG;
    }
    fbim_handle h = new (std::nothrow) fbim_handle_s();
    if (!h) return FBIM_ERR_OOM;
    fbim_status st = guarded(h, [&]() -> fbim_status {
        h->n_b = n_b;
        h->n_p = n_p;
        h->N = n_b * n_p;
        h->L = L;
        h->tol = tol;
        h->eta = p.eta > 0 ? p.eta : 1.0;
        h->order = p.alpert_order ? p.alpert_order : 4;
        h->precision = p.precision;
        h->device = p.device;
        h->restart = p.restart > 0 ? p.restart : 60;
        h->autotune = p.autotune;
        h->tensor_cores = p.tensor_cores;
        h->stream = (cudaStream_t)p.stream;
        FBIM_CUDA_TRY(h, cudaSetDevice(h->device));
        FBIM_CUDA_TRY(h, cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
        FBIM_CUDA_TRY(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        FBIM_CUDA_TRY(h, cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
        h->host_ref.assign(ref_nodes_host, ref_nodes_host + 2 * n_p);
        for (int i = 0; i < 3 * n_b; ++i)
            if (!std::isfinite(Q_host[i])) {
                h->fail("non-finite body coordinates");
                return FBIM_ERR_NONFINITE;
            }
        FBIM_CUDA_TRY(h, cudaSetDevice(h->device));
        // the end-correction rule fixes the band; r_c defaults to r_Alpert / 0.6 (Sec. 4.1)
        std::vector<double> v, w;
        int a;
        std::string err;
        if (fbim::alpert_rule(h->order, v, w, a, err) != FBIM_OK) {
            h->fail(err);
            return FBIM_ERR_SETUP;
        }
        int band = a - 1;
        for (double vk : v) band = std::max(band, (int)std::floor(vk) + (h->order + 2) / 2);
        if (2 * band + 1 > n_p) {
            h->fail("n_p too small for the Alpert correction band");
            return FBIM_ERR_INVALID_ARG;
        }
        double r_alpert = 0;
        for (int i = 0; i < n_p; ++i) {
            int k = (i + band) % n_p;
            double dx = ref_nodes_host[2 * i] - ref_nodes_host[2 * k];
            double dy = ref_nodes_host[2 * i + 1] - ref_nodes_host[2 * k + 1];
            r_alpert = std::max(r_alpert, std::sqrt(dx * dx + dy * dy));
        }
        double rc_req = r_c > 0 ? r_c : r_alpert / 0.6;
        if (rc_req > L / 3) rc_req = L / 3;
        int nbox, M, P;
        double rc, xx, es;
        if (fbim::choose_ewald(L, rc_req, tol, xi, nbox, rc, xx, M, P, es, err) != FBIM_OK) {
            h->fail(err);
            return FBIM_ERR_INVALID_ARG;
        }
        if (p.support > 0) P = p.support | 1;
        h->M_min = M;
        if (p.grid > 0) {
            M = p.grid + (p.grid & 1);
        } else if (p.grid_tune) {
            FBIM_CUDA_TRY(h, cudaSetDevice(h->device));
            h->precision = p.precision;
            FBIM_TRY(fbim::tune_grid(h, M, P, M, h->grid_tune_ms));
        }
        // wave-space tiles: TS divides M, TS <= 64, and a node's window (P - 1)/2 points
        // to each side never reaches past the neighbouring tile
        auto tile_side = [](int m) {
            int best = 0;
            for (int d = 1; d <= 64 && d <= m; ++d)
                if (m % d == 0) best = d;
            return best;
        };
        int TS = tile_side(M);
        while (TS < std::max(16, (P - 1) / 2) && TS < M) {
            if (p.grid > 0) {
                h->fail("grid side must have a divisor in [16, 64] (wave-space tiling)");
                return FBIM_ERR_INVALID_ARG;
            }
            M += 2;
            while (true) {
                int r = M;
                for (int f : {2, 3, 5, 7})
                    while (r % f == 0) r /= f;
                if (r == 1) break;
                M += 2;
            }
            TS = tile_side(M);
        }
        h->TS = TS;
        h->n_tile = M / TS;
        h->n_box = nbox;
        // FP32 operator: its own support on the same grid (the support rule at the
        // larger of tol and 1e-7), the Gaussian shape following it
        {
            int P32 = p.fp32_support > 0 ? (p.fp32_support | 1)
                                         : (int)std::ceil(2.0 * std::log(1.0 / std::max(tol, 1e-7)) / M_PI);
            if (P32 % 2 == 0) ++P32;
            h->P32 = p.precision == FBIM_FP32 ? std::max(3, std::min(P32, P)) : P;
        }
        h->r_c = rc;
        h->xi = xx;
        h->M = M;
        h->P = P;
        h->h = L / M;
        {
            double wdt = P * h->h / 2.0, m = std::sqrt(M_PI * P);
            h->eta_s = std::pow(2.0 * wdt * h->xi / m, 2);
            wdt = h->P32 * h->h / 2.0;
            m = std::sqrt(M_PI * h->P32);
            h->eta_s32 = std::pow(2.0 * wdt * h->xi / m, 2);
        }
        if (!(h->eta_s < 1.0) || P > M || P > 23) {
            h->fail("Gaussian support/grid inconsistent (need eta_s < 1, P <= min(M, 23), i.e. tol >= 1e-15)");
            return FBIM_ERR_INVALID_ARG;
        }
        std::vector<double> bandv;
        FBIM_TRY(fbim::alpert_reference_band(h, bandv));
        h->host_band = bandv;
        // Chebyshev series of the smooth part of E1 on [0, xi^2 r_c^2]
        h->zmax = h->xi * h->xi * h->r_c * h->r_c * (1.0 + 1e-6);
        {
            // one interpolant of degree kChebMax - 1, truncated per precision where its
            // coefficients fall below 1e-15 (FP64) or 1e-8 (FP32) of the largest: the
            // truncation error then sits below each precision's rounding
            std::vector<double> c;
            const int dmax = fbim::kChebMax - 1;
            fbim::e1_chebyshev(h->zmax, dmax, c);
            double cmax = 0;
            for (double v : c) cmax = std::max(cmax, std::fabs(v));
            auto degree = [&](double rel) {
                int d = dmax;
                while (d > 4 && std::fabs(c[d]) < rel * cmax) --d;
                return std::min(dmax, d + 1);
            };
            const int d64 = degree(1e-15), d32 = degree(1e-8);
            h->cheb64.deg = d64;
            h->cheb64.scale = 2.0 / h->zmax;
            for (int k = 0; k <= d64; ++k) h->cheb64.c[k] = c[k];
            h->cheb32.deg = d32;
            h->cheb32.scale = (float)(2.0 / h->zmax);
            for (int k = 0; k <= d32; ++k) h->cheb32.c[k] = (float)c[k];
        }
        const size_t N = h->N, nc = (size_t)h->n_cell();
        FBIM_CUDA_TRY(h, cudaMalloc(&h->ref, 2 * n_p * sizeof(double)));
        FBIM_CUDA_TRY(h, cudaMalloc(&h->Q, 3 * n_b * sizeof(double)));
        FBIM_CUDA_TRY(h, cudaMalloc(&h->x, 2 * N * sizeof(double)));
        FBIM_CUDA_TRY(h, cudaMalloc(&h->cell, N * sizeof(int)));
        FBIM_CUDA_TRY(h, cudaMalloc(&h->cell_start, fbim::scan_storage((int)nc) * sizeof(int)));
        FBIM_CUDA_TRY(h, cudaMalloc(&h->cell_fill, nc * sizeof(int)));
        FBIM_CUDA_TRY(h, cudaMalloc(&h->perm, N * sizeof(int)));
        FBIM_CUDA_TRY(h, cudaMalloc(&h->slot, N * sizeof(int)));
        FBIM_CUDA_TRY(h, cudaMalloc(&h->flags, 4 * sizeof(int)));
        FBIM_CUDA_TRY(h, cudaMalloc(&h->band_dev, bandv.size() * sizeof(double)));
        const size_t ntl = (size_t)h->n_tile * h->n_tile;
        FBIM_CUDA_TRY(h, cudaMalloc(&h->gbase, N * sizeof(int2)));
        FBIM_CUDA_TRY(h, cudaMalloc(&h->tile_start, fbim::scan_storage((int)ntl) * sizeof(int)));
        FBIM_CUDA_TRY(h, cudaMalloc(&h->tile_fill, ntl * sizeof(int)));
        FBIM_CUDA_TRY(h, cudaMalloc(&h->tperm, N * sizeof(int)));
        FBIM_CUDA_TRY(h, cudaMalloc(&h->tslot, N * sizeof(int)));
        FBIM_CUDA_TRY(h, cudaMalloc(&h->tile_tmp, N * sizeof(int)));
        FBIM_CUDA_TRY(h, cudaMalloc(&h->rot, 2 * n_b * sizeof(double)));
        FBIM_CUDA_TRY(h, cudaMemsetAsync(h->flags, 0, 4 * sizeof(int), h->stream));
        FBIM_CUDA_TRY(h, cudaMemcpyAsync(h->ref, ref_nodes_host, 2 * n_p * sizeof(double), cudaMemcpyHostToDevice,
                                         h->stream));
        FBIM_CUDA_TRY(h, cudaMemcpyAsync(h->Q, Q_host, 3 * n_b * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        FBIM_CUDA_TRY(h, cudaMemcpyAsync(h->band_dev, bandv.data(), bandv.size() * sizeof(double),
                                         cudaMemcpyHostToDevice, h->stream));
        FBIM_TRY(fbim::build_geometry(h));
        if (h->precision == FBIM_FP32) FBIM_TRY(fbim::ensure_ewald<float>(h));
        FBIM_TRY(fbim::ensure_ewald<double>(h));
        FBIM_TRY(fbim::noalloc_prepare(h));
        return check_flags(h);
    });
    if (st != FBIM_OK) {
        set_global_error(h->err);
        release(h);
        return st;
    }
    *out = h;
    return FBIM_OK;
}

// Split tuner.  The Ewald split parameter moves work between the real-space pair
// sum (grows with r_c^2) and the wave space (the grid side shrinks like 1/r_c); with
// the pair sum running beside the wave-space chain the best r_c is found by timing.
// Candidates r_c >= the given one (the Alpert band sets its lower bound), each on a
// throwaway handle: cost = 25 FP32 operator applications + 1 FP64 residual
// application + 1 geometry update (one mixed-precision solve), or 25 FP64
// applications + 1 update for an FP64 handle.
static fbim_status tune_split(int n_b, int n_p, const double* ref, const double* Q, double L, double r_c0, double tol,
                              fbim_params p, double& r_best, int& n_cand, double& best_ms) {
    p.split_tune = 0;
    r_best = r_c0;
    n_cand = 0;
    best_ms = 0;
    const bool f32 = p.precision == FBIM_FP32;
    double best = 1e300;
    int last_box = -1;
    for (double fac : {1.0, 1.25, 1.5, 1.8, 2.2}) {
        const double rc = std::min(r_c0 * fac, L / 3.0);
        const int nbox = std::max(3, (int)std::floor(L / rc));
        if (nbox == last_box) continue;
        last_box = nbox;
        fbim_handle h = nullptr;
        if (setup_one(&h, n_b, n_p, ref, Q, L, L / nbox, 0.0, tol, &p) != FBIM_OK) continue;
        double* buf = nullptr;
        const size_t N = (size_t)h->N;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        bool ok = cudaMalloc(&buf, 2 * 2 * N * sizeof(double)) == cudaSuccess &&
                  cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
                  cudaMemsetAsync(buf, 0, 2 * N * sizeof(double), h->stream) == cudaSuccess;
        double* mu = buf;
        double* v = buf + 2 * N;
        auto timeit = [&](int warm, int reps, auto&& fn) -> double {
            for (int r = 0; r < warm && ok; ++r) ok = fn() == FBIM_OK;
            cudaEventRecord(e0, h->stream);
            for (int r = 0; r < reps && ok; ++r) ok = fn() == FBIM_OK;
            cudaEventRecord(e1, h->stream);
            float ms = 0.f;
            ok = ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            return ms / reps;
        };
        // a non-zero force on every node (the cost does not depend on the values)
        if (ok) ok = cudaMemcpyAsync(mu, h->Q, sizeof(double) * std::min<size_t>(2 * N, 3 * (size_t)n_b),
                                     cudaMemcpyDeviceToDevice, h->stream) == cudaSuccess;
        const double t_lo = f32 ? timeit(2, 5, [&] { return fbim_apply_stokeslet(h, mu, v); }) : 0.0;
        const double t_hi = timeit(1, f32 ? 2 : 5, [&] { return fbim_apply_stokeslet_fp64(h, mu, v); });
        const double t_up = timeit(1, 2, [&] { return fbim_update_config(h, h->Q); });
        const double cost = f32 ? 25.0 * t_lo + t_hi + t_up : 25.0 * t_hi + t_up;
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(buf);
        fbim_destroy(h);
        cudaGetLastError();
        if (!ok) continue;
        ++n_cand;
        if (cost < best) {
            best = cost;
            r_best = L / nbox;
        }
    }
    best_ms = best < 1e300 ? best : 0.0;
    return n_cand > 0 ? FBIM_OK : FBIM_ERR_SETUP;
}

extern "C" fbim_status fbim_setup(fbim_handle* out, int n_b, int n_p, const double* ref_nodes_host,
                                  const double* Q_host, double L, double r_c, double xi, double tol,
                                  const fbim_params* opt) {
    fbim_params p;
    fbim_default_params(&p);
    if (opt) p = *opt;
    if (!p.split_tune || !(r_c > 0) || !out || !(L > 0) || !(tol > 0 && tol < 1) || n_b <= 0 || n_p < 8 ||
        !ref_nodes_host || !Q_host)
        return setup_one(out, n_b, n_p, ref_nodes_host, Q_host, L, r_c, xi, tol, opt);
    double r_best = r_c, cost = 0;
    int n_cand = 0;
    if (tune_split(n_b, n_p, ref_nodes_host, Q_host, L, r_c, tol, p, r_best, n_cand, cost) != FBIM_OK)
        r_best = r_c;  // tuning is optional: fall back to the given cutoff
    p.split_tune = 0;
    const fbim_status st = setup_one(out, n_b, n_p, ref_nodes_host, Q_host, L, r_best, n_cand > 0 ? 0.0 : xi, tol, &p);
    if (st == FBIM_OK) {
        (*out)->split_candidates = n_cand;
        (*out)->split_cost_ms = cost;
    }
    return st;
}

extern "C" fbim_status fbim_update_config(fbim_handle h, const double* Q_dev) {
    if (!h || !Q_dev) return FBIM_ERR_INVALID_ARG;
    return guarded(h, [&]() -> fbim_status {
        FBIM_CUDA_TRY(h, cudaSetDevice(h->device));
        FBIM_TRY(fbim::update_positions(h, Q_dev));
        return check_flags(h);
    });
}

namespace {
__global__ void k_displaced(int n, const double* __restrict__ Q, double a, const double* __restrict__ W,
                            double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = Q[i] + a * W[i];
}
}  // namespace

extern "C" fbim_status fbim_update_config_displaced(fbim_handle h, const double* Q_dev, double a, const double* W_dev) {
    if (!h || !Q_dev || !W_dev || !std::isfinite(a)) return FBIM_ERR_INVALID_ARG;
    return guarded(h, [&]() -> fbim_status {
        FBIM_CUDA_TRY(h, cudaSetDevice(h->device));
        const int n = 3 * h->n_b;
        // Q_dev or W_dev may be the handle's own coordinates: the sum is elementwise
        k_displaced<<<(n + 255) / 256, 256, 0, h->stream>>>(n, Q_dev, a, W_dev, h->Q);
        h->launches += 1;
        FBIM_CUDA_TRY(h, cudaGetLastError());
        FBIM_TRY(fbim::update_positions(h, h->Q));
        return check_flags(h);
    });
}

static fbim_status apply_which(fbim_handle h, const double* mu, double* v, int which, bool fp64 = false) {
    if (!h || !mu || !v) return FBIM_ERR_INVALID_ARG;
    if ((((uintptr_t)mu) | ((uintptr_t)v)) & 15) {
        h->fail("mu and v must be 16-byte aligned");
        return FBIM_ERR_INVALID_ARG;
    }
    return guarded(h, [&]() -> fbim_status {
        FBIM_CUDA_TRY(h, cudaSetDevice(h->device));
        if (h->precision == FBIM_FP32 && !fp64) return fbim::apply_operator<float>(h, mu, v, which);
        return fbim::apply_operator<double>(h, mu, v, which);
    });
}

extern "C" fbim_status fbim_apply_stokeslet_fp64(fbim_handle h, const double* mu_dev, double* v_dev) {
    return apply_which(h, mu_dev, v_dev, 3, true);
}

extern "C" fbim_status fbim_apply_stokeslet(fbim_handle h, const double* mu_dev, double* v_dev) {
    return apply_which(h, mu_dev, v_dev, 3);
}

extern "C" fbim_status fbim_apply_real(fbim_handle h, const double* mu_dev, double* v_dev) {
    return apply_which(h, mu_dev, v_dev, 1);
}

extern "C" fbim_status fbim_apply_wave(fbim_handle h, const double* mu_dev, double* v_dev) {
    return apply_which(h, mu_dev, v_dev, 2);
}

extern "C" fbim_status fbim_get_info(fbim_handle h, fbim_info* info) {
    if (!h || !info) return FBIM_ERR_INVALID_ARG;
    info->n_b = h->n_b;
    info->n_p = h->n_p;
    info->n_nodes = h->N;
    info->L = h->L;
    info->xi = h->xi;
    info->r_c = h->r_c;
    info->tol = h->tol;
    info->n_box = h->n_box;
    info->grid = h->M;
    info->support = h->P;
    info->eta_s = h->eta_s;
    info->support32 = h->P32;
    info->eta_s32 = h->eta_s32;
    info->h = h->h;
    info->alpert_order = h->order;
    info->alpert_nodes = h->aj;
    info->alpert_window = h->aa;
    info->alpert_band = h->band;
    info->precision = h->precision;
    info->tile = h->TS;
    const bool f32 = h->precision == FBIM_FP32;
    info->pair_entries = f32 ? h->e32.n_padded : h->e64.n_padded;
    info->wave_variant = f32 ? h->e32.spread_variant : h->e64.spread_variant;
    info->interp_variant = f32 ? h->e32.interp_variant : h->e64.interp_variant;
    for (int v = 0; v < 2; ++v) {
        info->variant_ms[v] = f32 ? h->e32.variant_ms[0][v] : h->e64.variant_ms[0][v];
        info->interp_ms[v] = f32 ? h->e32.variant_ms[1][v] : h->e64.variant_ms[1][v];
    }
    info->launches = h->launches;
    info->grid_min = h->M_min;
    info->grid_tune_ms = h->grid_tune_ms;
    info->split_candidates = h->split_candidates;
    info->split_cost_ms = h->split_cost_ms;
    info->fp64_fft = h->precision == FBIM_FP32 ? h->fft64.state : -1;
    info->coarse_fallbacks = h->coarse_fallbacks;
    return FBIM_OK;
}

extern "C" void fbim_destroy(fbim_handle h) { release(h); }

extern "C" const char* fbim_last_error(fbim_handle h) { return h ? h->err.c_str() : fbim::global_error(); }

// ---------------------------------------------------------------------------
// Stage timing
// ---------------------------------------------------------------------------
void fbim_handle_s::mark_begin() {
    if (!timing) return;
    cudaEventRecord(ev[0], stream);
    n_ev = 1;
}

void fbim_handle_s::mark(int stage) {
    if (!timing || n_ev <= 0 || n_ev >= 16) return;
    cudaEventRecord(ev[n_ev], stream);
    ev_stage[n_ev] = stage;
    ++n_ev;
}

void fbim_handle_s::collect() {
    if (!timing || n_ev < 2) return;
    cudaEventSynchronize(ev[n_ev - 1]);
    for (int i = 1; i < n_ev; ++i) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[i - 1], ev[i]);
        stage_ms[ev_stage[i]] += ms;
        stage_calls[ev_stage[i]] += 1;
    }
    n_ev = 0;
}

extern "C" fbim_status fbim_set_timing(fbim_handle h, int on) {
    if (!h) return FBIM_ERR_INVALID_ARG;
    return guarded(h, [&]() -> fbim_status {
        FBIM_CUDA_TRY(h, cudaSetDevice(h->device));
        if (on && !h->ev[0])
            for (auto& e : h->ev) FBIM_CUDA_TRY(h, cudaEventCreate(&e));
        h->timing = on != 0;
        for (int i = 0; i < FBIM_N_STAGES; ++i) {
            h->stage_ms[i] = 0;
            h->stage_calls[i] = 0;
        }
        h->n_ev = 0;
        return FBIM_OK;
    });
}

extern "C" fbim_status fbim_stage_times(fbim_handle h, double* ms, long long* calls, int n) {
    if (!h || !ms || n <= 0) return FBIM_ERR_INVALID_ARG;
    for (int i = 0; i < n && i < FBIM_N_STAGES; ++i) {
        ms[i] = h->stage_ms[i];
        if (calls) calls[i] = h->stage_calls[i];
    }
    return FBIM_OK;
}
