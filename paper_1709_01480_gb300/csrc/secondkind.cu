// Completed second-kind (double-layer) mobility solver (App. B, Eqs. DLrepresentation,
// second-kind-formulation, q2torque): the reference solver of the paper, FP64 throughout.
//
// Unknowns x = [phi (2N); U (3 N_b)], the layout of the first-kind saddle vector.  The
// operator A x has node rows
//     u_b + omega_b (x - q_b)^perp - 1/2 phi - (D phi)
// and closure rows |Gamma| u_b - sum phi ds, W omega_b - sum phi . (x - q_b)^perp ds;
// the right-hand side is [C F; 0], C F the periodic Stokeslets and rotlets of the
// bodies' forces and torques at every node.  D is the periodic double layer with
// S_lm = phi_l n_m ds (n into the body), split as App. B prints it:
//   * real space: T^(r) over the cell list (pairs within r_c, minimum image), the
//     trapezoidal self term -(1/4 pi) 2 kappa (t t^T) phi ds replacing the s = t entry;
//   * wave space: the four fields S_lm spread with the Gaussian window of the handle's
//     FP64 operator, one batched D2Z, the stresslet multiplier -i T^(w)_jlm / (4 pi)
//     (its e^{-k^2/4xi^2} split into the two windows and e^{-(1-eta_s) k^2/4xi^2}),
//     one batched Z2D, interpolation;
//   * the mean-flow term (1/V) sum_s x_s (phi_s . n_s) ds_s at every node.
// The completion uses the same machinery (real-space Stokeslet and rotlet within r_c of
// each tracking point, three wave fields f_x, f_y, tau spread at the tracking points).
// GMRES without preconditioning (App. B: the formulation is well conditioned), FP64
// classical Gram-Schmidt twice on the device.
//
// The readings of App. B that this follows (normal into the body, the rotlet's
// 1/(4 pi eta V), T^(0) at the source position, the weighted self term, counter-
// clockwise perp) are those of the oracle's restatement of App. B.
#include <cufft.h>

#include <cmath>
#include <vector>

#include "ewald_types.cuh"
#include "fbim_internal.h"
#include "solver.cuh"

struct SecondKind {
    unsigned long long geom = ~0ull;    // geometry version the per-node arrays were built for
    int M = 0, Mh = 0;
    cufftHandle plan_f4 = 0, plan_f3 = 0, plan_i2 = 0;
    double* grid = nullptr;             // [4][M][M] spread fields, then [2][M][M] velocities
    cufftDoubleComplex* spec = nullptr; // [4][M][Mh]
    double* tn_ref = nullptr;           // [n_p][6]: tangent, inward normal, ds, kappa
    double4* tn = nullptr;              // [N] (t_x, t_y, n_x, n_y), body order
    double2* xu = nullptr;              // [N] q_b + R_b gamma_ref (unwrapped positions)
    double2* rel = nullptr;             // [N] R_b gamma_ref = x - q_b
    double* bsum = nullptr;             // [n_b][5] per-body sums
    double* cmean = nullptr;            // [2] mean-flow velocity
    double len = 0, W = 0;              // |Gamma| and int |x - q|^2 dS (the same for every body)
    // GMRES workspace
    int m = 0;
    double* V = nullptr;                // [m + 1][ld] basis
    double* vin = nullptr;              // [ld] operator input
    double* w = nullptr;                // [ld] operator output
    double* b = nullptr;                // [ld] right-hand side
    double* r = nullptr;                // [ld] residual
    double* y = nullptr;                // [m] combination coefficients (device)
    double* sf = nullptr;               // [N][4] S_lm per node
    double* qw = nullptr;               // [n_b][2] tracking points wrapped into the box
    CgsState cgs;
};

namespace fbim {

namespace {

constexpr double kInv4Pi = 0.07957747154594766788;  // 1 / (4 pi)

// per-node geometry: rotated tangent and inward normal, unwrapped position, x - q
__global__ void k_sk_geom(int N, int n_p, const double* __restrict__ Q, const double* __restrict__ rot,
                          const double* __restrict__ ref, const double* __restrict__ tn_ref,
                          double4* __restrict__ tn, double2* __restrict__ xu, double2* __restrict__ rel) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    const int b = m / n_p, j = m - b * n_p;
    const double c = rot[2 * b], s = rot[2 * b + 1];
    const double* g = tn_ref + 6 * j;
    tn[m] = make_double4(c * g[0] - s * g[1], s * g[0] + c * g[1], c * g[2] - s * g[3], s * g[2] + c * g[3]);
    const double gx = ref[2 * j], gy = ref[2 * j + 1];
    const double rx = c * gx - s * gy, ry = s * gx + c * gy;
    rel[m] = make_double2(rx, ry);
    xu[m] = make_double2(Q[3 * b] + rx, Q[3 * b + 1] + ry);
}

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

// per body (one block each): sum phi ds (2), sum phi . (x - q)^perp ds, sum x_s (phi . n) ds (2)
__global__ void k_sk_body_sums(int n_p, const double* __restrict__ phi, const double4* __restrict__ tn,
                               const double2* __restrict__ xu, const double2* __restrict__ rel,
                               const double* __restrict__ tn_ref, double* __restrict__ bsum) {
    __shared__ double red[32];
    const int b = blockIdx.x;
    double a[5] = {0, 0, 0, 0, 0};
    for (int j = threadIdx.x; j < n_p; j += blockDim.x) {
        const int m = b * n_p + j;
        const double ds = tn_ref[6 * j + 4];
        const double px = phi[2 * m], py = phi[2 * m + 1];
        const double2 r = rel[m];
        const double4 t = tn[m];
        const double pn = px * t.z + py * t.w;
        a[0] += px * ds;
        a[1] += py * ds;
        a[2] += (-r.y * px + r.x * py) * ds;
        a[3] += xu[m].x * pn * ds;
        a[4] += xu[m].y * pn * ds;
    }
    for (int q = 0; q < 5; ++q) {
        const double s = block_sum(a[q], red);
        if (threadIdx.x == 0) bsum[5 * b + q] = s;
    }
}

// mean-flow velocity c = (1/V) sum_b sum_s x_s (phi . n) ds (one block, fixed order)
__global__ void k_sk_mean(int n_b, double inv_V, const double* __restrict__ bsum, double* __restrict__ cmean) {
    __shared__ double red[32];
    double cx = 0, cy = 0;
    for (int b = threadIdx.x; b < n_b; b += blockDim.x) {
        cx += bsum[5 * b + 3];
        cy += bsum[5 * b + 4];
    }
    const double sx = block_sum(cx, red);
    if (threadIdx.x == 0) cmean[0] = sx * inv_V;
    const double sy = block_sum(cy, red);
    if (threadIdx.x == 0) cmean[1] = sy * inv_V;
}

// node rows without the double layer's pair and wave parts:
// y = u + omega (x - q)^perp - phi/2 + (1/4 pi) 2 kappa t (t . phi) ds - c
__global__ void k_sk_local(int N, int n_p, const double* __restrict__ x, const double4* __restrict__ tn,
                           const double2* __restrict__ rel, const double* __restrict__ tn_ref,
                           const double* __restrict__ cmean, double* __restrict__ y) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    const int b = m / n_p, j = m - b * n_p;
    const double* U = x + 2 * (size_t)N + 3 * b;
    const double2 r = rel[m];
    const double4 t = tn[m];
    const double ds = tn_ref[6 * j + 4], kap = tn_ref[6 * j + 5];
    const double px = x[2 * m], py = x[2 * m + 1];
    const double sf = 2.0 * kInv4Pi * kap * ds * (t.x * px + t.y * py);
    y[2 * m] = U[0] - U[2] * r.y - 0.5 * px + sf * t.x - cmean[0];
    y[2 * m + 1] = U[1] + U[2] * r.x - 0.5 * py + sf * t.y - cmean[1];
}

// closure rows |Gamma| u - sum phi ds, W omega - sum phi . (x - q)^perp ds
__global__ void k_sk_closure(int N, int n_b, double len, double W, const double* __restrict__ x,
                             const double* __restrict__ bsum, double* __restrict__ y) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_b) return;
    const double* U = x + 2 * (size_t)N + 3 * b;
    double* o = y + 2 * (size_t)N + 3 * b;
    o[0] = len * U[0] - bsum[5 * b];
    o[1] = len * U[1] - bsum[5 * b + 1];
    o[2] = W * U[2] - bsum[5 * b + 2];
}

// y_t -= sum_{s != t, |r| < r_c} T^(r)(x_t - x_s) : (phi_s n_s ds_s), minimum image over
// the 3 x 3 neighbouring cells (n_box >= 3)
__global__ void k_sk_real(int N, int n_p, int n_box, double L, double rc2, double xi2,
                          const double* __restrict__ xw, const int* __restrict__ cell,
                          const int* __restrict__ cell_start, const int* __restrict__ perm,
                          const double* __restrict__ phi, const double4* __restrict__ tn,
                          const double* __restrict__ tn_ref, double* __restrict__ y) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    const double xt = xw[2 * t], yt = xw[2 * t + 1];
    const int c = cell[t], cx = c % n_box, cy = c / n_box;
    double vx = 0, vy = 0;
    for (int dy = -1; dy <= 1; ++dy) {
        const int ny = (cy + dy + n_box) % n_box;
        for (int dx = -1; dx <= 1; ++dx) {
            const int nc = ny * n_box + (cx + dx + n_box) % n_box;
            for (int q = cell_start[nc]; q < cell_start[nc + 1]; ++q) {
                const int s = perm[q];
                if (s == t) continue;
                double rx = xt - xw[2 * s], ry = yt - xw[2 * s + 1];
                rx -= L * rint(rx / L);
                ry -= L * rint(ry / L);
                const double r2 = rx * rx + ry * ry;
                if (r2 >= rc2) continue;
                const double ds = tn_ref[6 * (s % n_p) + 4];
                const double4 g = tn[s];
                const double px = phi[2 * s] * ds, py = phi[2 * s + 1] * ds;
                const double z = xi2 * r2, e = exp(-z);
                const double rp = rx * px + ry * py, rn = rx * g.z + ry * g.w, pn = px * g.z + py * g.w;
                const double a = -4.0 * rp * rn * (1.0 + z) / (r2 * r2);
                const double bq = 2.0 * xi2;
                vx += e * (a * rx + bq * (rx * pn + g.z * rp));
                vy += e * (a * ry + bq * (ry * pn + g.w * rp));
            }
        }
    }
    y[2 * t] -= kInv4Pi * vx;
    y[2 * t + 1] -= kInv4Pi * vy;
}

// Gaussian window g(d) = (2 xi^2 / (pi eta_s)) exp(-(2 xi^2 / eta_s) |d|^2), P x P grid points
// around the nearest one.  Spread: one block per source, the window's points over the
// threads, FP64 atomics into the F fields [F][M][M].
template <int F>
__global__ void k_sk_spread(int n_src, const double* __restrict__ pos, int pos_stride,
                            const double* __restrict__ val, int val_stride, int M, int P, double h, double a,
                            double g0, double* __restrict__ grid) {
    const int s = blockIdx.x;
    if (s >= n_src) return;
    const double px = pos[(size_t)pos_stride * s], py = pos[(size_t)pos_stride * s + 1];
    const double fx = px / h, fy = py / h;
    const int ix0 = (int)floor(fx + 0.5), iy0 = (int)floor(fy + 0.5);
    const int hw = (P - 1) / 2;
    double v[F];
#pragma unroll
    for (int f = 0; f < F; ++f) v[f] = val[(size_t)val_stride * s + f];
    const size_t MM = (size_t)M * M;
    for (int k = threadIdx.x; k < P * P; k += blockDim.x) {
        const int oy = k / P - hw, ox = k % P - hw;
        const double dx = (fx - (ix0 + ox)) * h, dy = (fy - (iy0 + oy)) * h;
        const double wgt = g0 * exp(-a * (dx * dx + dy * dy));
        int gx = (ix0 + ox) % M, gy = (iy0 + oy) % M;
        gx += gx < 0 ? M : 0;
        gy += gy < 0 ? M : 0;
        const size_t o = (size_t)gy * M + gx;
#pragma unroll
        for (int f = 0; f < F; ++f) atomicAdd(grid + f * MM + o, wgt * v[f]);
    }
}

// Interpolation: one block per target, out[2 t + c] += sign * sum_window g G_c (c = 0, 1)
__global__ void k_sk_interp(int n_tgt, const double* __restrict__ pos, int M, int P, double h, double a, double g0,
                            const double* __restrict__ grid, double sign, double* __restrict__ out) {
    __shared__ double red[32];
    const int t = blockIdx.x;
    if (t >= n_tgt) return;
    const double px = pos[2 * (size_t)t], py = pos[2 * (size_t)t + 1];
    const double fx = px / h, fy = py / h;
    const int ix0 = (int)floor(fx + 0.5), iy0 = (int)floor(fy + 0.5);
    const int hw = (P - 1) / 2;
    const size_t MM = (size_t)M * M;
    double u0 = 0, u1 = 0;
    for (int k = threadIdx.x; k < P * P; k += blockDim.x) {
        const int oy = k / P - hw, ox = k % P - hw;
        const double dx = (fx - (ix0 + ox)) * h, dy = (fy - (iy0 + oy)) * h;
        const double wgt = g0 * exp(-a * (dx * dx + dy * dy));
        int gx = (ix0 + ox) % M, gy = (iy0 + oy) % M;
        gx += gx < 0 ? M : 0;
        gy += gy < 0 ? M : 0;
        const size_t o = (size_t)gy * M + gx;
        u0 += wgt * grid[o];
        u1 += wgt * grid[MM + o];
    }
    const double s0 = block_sum(u0, red);
    const double s1 = block_sum(u1, red);
    if (threadIdx.x == 0) {
        out[2 * (size_t)t] += sign * s0;
        out[2 * (size_t)t + 1] += sign * s1;
    }
}

// S_lm = phi_l n_m ds per node, field f = l + 2 m
__global__ void k_sk_sfields(int N, int n_p, const double* __restrict__ phi, const double4* __restrict__ tn,
                             const double* __restrict__ tn_ref, double* __restrict__ S) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    const double ds = tn_ref[6 * (m % n_p) + 4];
    const double4 g = tn[m];
    const double px = phi[2 * m] * ds, py = phi[2 * m + 1] * ds;
    S[4 * m] = px * g.z;
    S[4 * m + 1] = py * g.z;
    S[4 * m + 2] = px * g.w;
    S[4 * m + 3] = py * g.w;
}

__device__ __forceinline__ bool sk_mode(int i, int M, int Mh, double twopi_L, double& kx, double& ky) {
    const int r = i / Mh, c = i - r * Mh;
    if ((r == 0 && c == 0) || c == M / 2 || r == M / 2) return false;  // zero mode and Nyquist lines
    kx = twopi_L * c;
    ky = twopi_L * (r <= M / 2 ? r : r - M);
    return true;
}

// stresslet multiplier on the four spectra S^_lm (fields l + 2m) -> two velocity spectra
// (in fields 0, 1): u^_j = scale (i E / k^4) [hk (k^2 (k_j tr S^ + (k^T S^)_j) - 2 k_j k^T S^ k) + k^2 (S^ k)_j]
__global__ void k_sk_scale_T(int M, int Mh, double twopi_L, double inv4xi2, double one_m_eta, double scale,
                             cufftDoubleComplex* __restrict__ spec) {
    const size_t n = (size_t)M * Mh;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double kx, ky;
    if (!sk_mode((int)i, M, Mh, twopi_L, kx, ky)) {
        spec[i] = make_cuDoubleComplex(0.0, 0.0);
        spec[n + i] = make_cuDoubleComplex(0.0, 0.0);
        return;
    }
    const double k2 = kx * kx + ky * ky;
    const double hk = 1.0 + k2 * inv4xi2, E = exp(-one_m_eta * k2 * inv4xi2);
    const cufftDoubleComplex s11 = spec[i], s21 = spec[n + i], s12 = spec[2 * n + i], s22 = spec[3 * n + i];
    double out[2][2];  // [j][re, im]
    for (int part = 0; part < 2; ++part) {
        const double S11 = part ? s11.y : s11.x, S21 = part ? s21.y : s21.x;
        const double S12 = part ? s12.y : s12.x, S22 = part ? s22.y : s22.x;
        const double tr = S11 + S22;
        const double kS1 = kx * S11 + ky * S21, kS2 = kx * S12 + ky * S22;   // (k^T S)_j
        const double Sk1 = S11 * kx + S12 * ky, Sk2 = S21 * kx + S22 * ky;   // (S k)_j
        const double kSk = kx * Sk1 + ky * Sk2;
        out[0][part] = hk * (k2 * (kx * tr + kS1) - 2.0 * kx * kSk) + k2 * Sk1;
        out[1][part] = hk * (k2 * (ky * tr + kS2) - 2.0 * ky * kSk) + k2 * Sk2;
    }
    const double f = scale * E / (k2 * k2);
    // multiply by i f: (re, im) -> (-f im, f re)
    spec[i] = make_cuDoubleComplex(-f * out[0][1], f * out[0][0]);
    spec[n + i] = make_cuDoubleComplex(-f * out[1][1], f * out[1][0]);
}

// Stokeslet and rotlet multipliers on the spectra of f_x, f_y, tau -> two velocity spectra:
// u^ = scale [hk E / k^2 (I - k^ k^^T) f^ - (i/2) k^perp hk E / k^2 tau^]
__global__ void k_sk_scale_GR(int M, int Mh, double twopi_L, double inv4xi2, double one_m_eta, double scale,
                              cufftDoubleComplex* __restrict__ spec) {
    const size_t n = (size_t)M * Mh;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double kx, ky;
    if (!sk_mode((int)i, M, Mh, twopi_L, kx, ky)) {
        spec[i] = make_cuDoubleComplex(0.0, 0.0);
        spec[n + i] = make_cuDoubleComplex(0.0, 0.0);
        return;
    }
    const double k2 = kx * kx + ky * ky;
    const double s = scale * (1.0 + k2 * inv4xi2) * exp(-one_m_eta * k2 * inv4xi2) / k2;
    const cufftDoubleComplex f1 = spec[i], f2 = spec[n + i], ta = spec[2 * n + i];
    const double a11 = 1.0 - kx * kx / k2, a22 = 1.0 - ky * ky / k2, a12 = -kx * ky / k2;
    // rotlet: -(i/2) k^perp tau^, k^perp = (-k_y, k_x); -(i/2) c (re, im) = (c im / 2, -c re / 2)
    const double r1 = -ky, r2 = kx;
    spec[i] = make_cuDoubleComplex(s * (a11 * f1.x + a12 * f2.x + 0.5 * r1 * ta.y),
                                   s * (a11 * f1.y + a12 * f2.y - 0.5 * r1 * ta.x));
    spec[n + i] = make_cuDoubleComplex(s * (a12 * f1.x + a22 * f2.x + 0.5 * r2 * ta.y),
                                       s * (a12 * f1.y + a22 * f2.y - 0.5 * r2 * ta.x));
}

// real-space completion: b_t = sum_b [G^(r)(x_t - q_b) f_b + R^(r)(x_t - q_b) tau_b] within r_c
// (pref = 1/(4 pi eta))
__global__ void k_sk_completion_real(int N, int n_b, double L, double rc2, double xi2, double pref,
                                     ChebE1<double> ce, const double* __restrict__ xw, const double* __restrict__ Q,
                                     const double* __restrict__ F, double* __restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    double vx = 0, vy = 0;
    for (int b = 0; b < n_b; ++b) {
        double qx = Q[3 * b] - L * floor(Q[3 * b] / L), qy = Q[3 * b + 1] - L * floor(Q[3 * b + 1] / L);
        double rx = xw[2 * t] - qx, ry = xw[2 * t + 1] - qy;
        rx -= L * rint(rx / L);
        ry -= L * rint(ry / L);
        const double r2 = rx * rx + ry * ry;
        if (r2 >= rc2 || r2 == 0.0) continue;
        const double z = xi2 * r2, e = exp(-z);
        const double a = kernel_a(ce, z), bb = e / r2;
        const double fx = F[3 * b], fy = F[3 * b + 1], tau = F[3 * b + 2];
        const double rf = rx * fx + ry * fy;
        const double rot = (1.0 - z) * e / r2 * tau;
        vx += a * fx + bb * rx * rf - ry * rot;
        vy += a * fy + bb * ry * rf + rx * rot;
    }
    out[2 * t] = pref * vx;
    out[2 * t + 1] = pref * vy;
}

// tracking points wrapped into the box (spread positions) and the zero closure rows
__global__ void k_sk_track(int n_b, double L, const double* __restrict__ Q, double* __restrict__ qw) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_b) return;
    qw[2 * b] = Q[3 * b] - L * floor(Q[3 * b] / L);
    qw[2 * b + 1] = Q[3 * b + 1] - L * floor(Q[3 * b + 1] / L);
}

}  // namespace

}  // namespace fbim

namespace fbim {

// Tangent, inward normal, ds and curvature of the reference curve by spectral
// differentiation of the trigonometric interpolant of its nodes (the Nyquist term of
// an even N_p contributes no derivative).
static void reference_curve(const std::vector<double>& ref, int n_p, std::vector<double>& tn, double& len,
                            double& W) {
    std::vector<double> d1(2 * n_p, 0.0), d2(2 * n_p, 0.0);
    std::vector<double> cr(2 * n_p), ci(2 * n_p);
    for (int k = 0; k < n_p; ++k)
        for (int c = 0; c < 2; ++c) {
            double sr = 0, si = 0;
            for (int j = 0; j < n_p; ++j) {
                const double a = -2.0 * M_PI * (double)j * k / n_p;
                sr += ref[2 * j + c] * std::cos(a);
                si += ref[2 * j + c] * std::sin(a);
            }
            cr[2 * k + c] = sr;
            ci[2 * k + c] = si;
        }
    for (int j = 0; j < n_p; ++j)
        for (int k = 0; k < n_p; ++k) {
            int kk = k <= n_p / 2 ? k : k - n_p;
            if (2 * k == n_p) kk = 0;
            const double a = 2.0 * M_PI * (double)j * k / n_p, ca = std::cos(a), sa = std::sin(a);
            for (int c = 0; c < 2; ++c) {
                const double re = cr[2 * k + c] * ca - ci[2 * k + c] * sa, im = cr[2 * k + c] * sa + ci[2 * k + c] * ca;
                d1[2 * j + c] += -kk * im / n_p;          // Re(i kk e)
                d2[2 * j + c] += -(double)kk * kk * re / n_p;
            }
        }
    tn.assign(6 * (size_t)n_p, 0.0);
    len = W = 0;
    for (int j = 0; j < n_p; ++j) {
        const double dx = d1[2 * j], dy = d1[2 * j + 1];
        const double sp = std::sqrt(dx * dx + dy * dy);
        const double tx = dx / sp, ty = dy / sp;
        const double ds = sp * 2.0 * M_PI / n_p;
        tn[6 * j] = tx;
        tn[6 * j + 1] = ty;
        tn[6 * j + 2] = -ty;   // inward normal: the outward one (t_y, -t_x) reversed
        tn[6 * j + 3] = tx;
        tn[6 * j + 4] = ds;
        tn[6 * j + 5] = (dx * d2[2 * j + 1] - dy * d2[2 * j]) / (sp * sp * sp);
        len += ds;
        W += (ref[2 * j] * ref[2 * j] + ref[2 * j + 1] * ref[2 * j + 1]) * ds;
    }
}

void free_second_kind(fbim_handle_s* h) {
    SecondKind* K = h->sk;
    if (!K) return;
    if (K->plan_f4) cufftDestroy(K->plan_f4);
    if (K->plan_f3) cufftDestroy(K->plan_f3);
    if (K->plan_i2) cufftDestroy(K->plan_i2);
    for (void* p : {(void*)K->grid, (void*)K->spec, (void*)K->tn_ref, (void*)K->tn, (void*)K->xu, (void*)K->rel,
                    (void*)K->bsum, (void*)K->cmean, (void*)K->V, (void*)K->vin, (void*)K->w, (void*)K->b,
                    (void*)K->r, (void*)K->y, (void*)K->sf, (void*)K->qw})
        cudaFree(p);
    cgs_free(K->cgs);
    delete K;
    h->sk = nullptr;
}

static fbim_status sk_setup(fbim_handle_s* h) {
    if (!h->sk) {
        if (h->n_box < 3) {
            h->fail("second-kind solver: needs at least 3 x 3 cells (r_c <= L/3)");
            return FBIM_ERR_INVALID_ARG;
        }
        SecondKind* K = new SecondKind();
        h->sk = K;
        const int N = h->N, n_b = h->n_b, M = h->M, Mh = M / 2 + 1;
        K->M = M;
        K->Mh = Mh;
        std::vector<double> tn;
        reference_curve(h->host_ref, h->n_p, tn, K->len, K->W);
        const size_t n = 2 * (size_t)N + 3 * n_b, ld = (n + 31) / 32 * 32;
        K->m = h->restart;
        FBIM_CUDA_TRY(h, cudaMalloc(&K->grid, sizeof(double) * 4 * (size_t)M * M));
        FBIM_CUDA_TRY(h, cudaMalloc(&K->spec, sizeof(cufftDoubleComplex) * 4 * (size_t)M * Mh));
        FBIM_CUDA_TRY(h, cudaMalloc(&K->tn_ref, sizeof(double) * tn.size()));
        FBIM_CUDA_TRY(h, cudaMalloc(&K->tn, sizeof(double4) * N));
        FBIM_CUDA_TRY(h, cudaMalloc(&K->xu, sizeof(double2) * N));
        FBIM_CUDA_TRY(h, cudaMalloc(&K->rel, sizeof(double2) * N));
        FBIM_CUDA_TRY(h, cudaMalloc(&K->bsum, sizeof(double) * 5 * n_b));
        FBIM_CUDA_TRY(h, cudaMalloc(&K->cmean, sizeof(double) * 2));
        FBIM_CUDA_TRY(h, cudaMalloc(&K->V, sizeof(double) * ld * (K->m + 1)));
        FBIM_CUDA_TRY(h, cudaMalloc(&K->vin, sizeof(double) * ld));
        FBIM_CUDA_TRY(h, cudaMalloc(&K->w, sizeof(double) * ld));
        FBIM_CUDA_TRY(h, cudaMalloc(&K->b, sizeof(double) * ld));
        FBIM_CUDA_TRY(h, cudaMalloc(&K->r, sizeof(double) * ld));
        FBIM_CUDA_TRY(h, cudaMalloc(&K->y, sizeof(double) * (K->m + 1)));
        FBIM_CUDA_TRY(h, cudaMalloc(&K->sf, sizeof(double) * 4 * (size_t)N));
        FBIM_CUDA_TRY(h, cudaMalloc(&K->qw, sizeof(double) * 2 * n_b));
        FBIM_CUDA_TRY(h, cudaMemcpyAsync(K->tn_ref, tn.data(), sizeof(double) * tn.size(), cudaMemcpyHostToDevice,
                                         h->stream));
        FBIM_TRY(cgs_alloc(h, K->cgs, (int)n, (int)ld, K->m));
        int dims[2] = {M, M};
        FBIM_CUFFT_TRY(h, cufftPlanMany(&K->plan_f4, 2, dims, nullptr, 1, M * M, nullptr, 1, M * Mh, CUFFT_D2Z, 4));
        FBIM_CUFFT_TRY(h, cufftPlanMany(&K->plan_f3, 2, dims, nullptr, 1, M * M, nullptr, 1, M * Mh, CUFFT_D2Z, 3));
        FBIM_CUFFT_TRY(h, cufftPlanMany(&K->plan_i2, 2, dims, nullptr, 1, M * Mh, nullptr, 1, M * M, CUFFT_Z2D, 2));
        FBIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    }
    SecondKind* K = h->sk;
    cufftSetStream(K->plan_f4, h->stream);
    cufftSetStream(K->plan_f3, h->stream);
    cufftSetStream(K->plan_i2, h->stream);
    if (K->geom != h->geom_version) {
        const int tb = 256;
        k_sk_geom<<<(h->N + tb - 1) / tb, tb, 0, h->stream>>>(h->N, h->n_p, h->Q, h->rot, h->ref, K->tn_ref, K->tn,
                                                             K->xu, K->rel);
        k_sk_track<<<(h->n_b + tb - 1) / tb, tb, 0, h->stream>>>(h->n_b, h->L, h->Q, K->qw);
        h->launches += 2;
        FBIM_CUDA_TRY(h, cudaGetLastError());
        K->geom = h->geom_version;
    }
    return FBIM_OK;
}

namespace {

struct SkWindow {
    double a, g0, twopi_L, inv4xi2, one_m_eta, scale;
};

SkWindow sk_window(const fbim_handle_s* h) {
    SkWindow w;
    const double xi2 = h->xi * h->xi;
    w.a = 2.0 * xi2 / h->eta_s;
    w.g0 = 2.0 * xi2 / (M_PI * h->eta_s);
    w.twopi_L = 2.0 * M_PI / h->L;
    w.inv4xi2 = 1.0 / (4.0 * xi2);
    w.one_m_eta = 1.0 - h->eta_s;
    const double hh = h->L / h->M;
    w.scale = hh * hh * hh * hh / (h->L * h->L);  // the double layer carries no viscosity
    return w;
}

}  // namespace

// y = A x (stream-ordered)
static fbim_status sk_apply(fbim_handle_s* h, const double* x, double* y) {
    SecondKind* K = h->sk;
    const int N = h->N, n_b = h->n_b, M = K->M, Mh = K->Mh, tb = 256;
    const double* phi = x;
    const SkWindow wd = sk_window(h);
    const double hh = h->L / M;
    k_sk_body_sums<<<n_b, 256, 0, h->stream>>>(h->n_p, phi, K->tn, K->xu, K->rel, K->tn_ref, K->bsum);
    k_sk_mean<<<1, 256, 0, h->stream>>>(n_b, 1.0 / (h->L * h->L), K->bsum, K->cmean);
    k_sk_local<<<(N + tb - 1) / tb, tb, 0, h->stream>>>(N, h->n_p, x, K->tn, K->rel, K->tn_ref, K->cmean, y);
    k_sk_closure<<<(n_b + tb - 1) / tb, tb, 0, h->stream>>>(N, n_b, K->len, K->W, x, K->bsum, y);
    k_sk_real<<<(N + 127) / 128, 128, 0, h->stream>>>(N, h->n_p, h->n_box, h->L, h->r_c * h->r_c, h->xi * h->xi,
                                                      h->x, h->cell, h->cell_start, h->perm, phi, K->tn, K->tn_ref,
                                                      y);
    // wave space of the double layer
    k_sk_sfields<<<(N + tb - 1) / tb, tb, 0, h->stream>>>(N, h->n_p, phi, K->tn, K->tn_ref, K->sf);
    FBIM_CUDA_TRY(h, cudaMemsetAsync(K->grid, 0, sizeof(double) * 4 * (size_t)M * M, h->stream));
    k_sk_spread<4><<<N, 128, 0, h->stream>>>(N, h->x, 2, K->sf, 4, M, h->P, hh, wd.a, wd.g0, K->grid);
    FBIM_CUFFT_TRY(h, cufftExecD2Z(K->plan_f4, K->grid, K->spec));
    const size_t ns = (size_t)M * Mh;
    k_sk_scale_T<<<(unsigned)((ns + tb - 1) / tb), tb, 0, h->stream>>>(M, Mh, wd.twopi_L, wd.inv4xi2, wd.one_m_eta,
                                                                       wd.scale, K->spec);
    FBIM_CUFFT_TRY(h, cufftExecZ2D(K->plan_i2, K->spec, K->grid));
    k_sk_interp<<<N, 128, 0, h->stream>>>(N, h->x, M, h->P, hh, wd.a, wd.g0, K->grid, -1.0, y);
    h->launches += 10;
    FBIM_CUDA_TRY(h, cudaGetLastError());
    return FBIM_OK;
}

// b = [C F; 0]: the periodic Stokeslets and rotlets of the tracking points at the nodes
static fbim_status sk_rhs(fbim_handle_s* h, const double* F, double* b) {
    SecondKind* K = h->sk;
    const int N = h->N, n_b = h->n_b, M = K->M, Mh = K->Mh, tb = 256;
    const SkWindow wd = sk_window(h);
    const double hh = h->L / M;
    k_sk_completion_real<<<(N + tb - 1) / tb, tb, 0, h->stream>>>(N, n_b, h->L, h->r_c * h->r_c, h->xi * h->xi,
                                                                 kInv4Pi / h->eta, h->cheb64, h->x, h->Q, F, b);
    FBIM_CUDA_TRY(h, cudaMemsetAsync(b + 2 * (size_t)N, 0, sizeof(double) * 3 * n_b, h->stream));
    FBIM_CUDA_TRY(h, cudaMemsetAsync(K->grid, 0, sizeof(double) * 3 * (size_t)M * M, h->stream));
    k_sk_spread<3><<<n_b, 128, 0, h->stream>>>(n_b, K->qw, 2, F, 3, M, h->P, hh, wd.a, wd.g0, K->grid);
    FBIM_CUFFT_TRY(h, cufftExecD2Z(K->plan_f3, K->grid, K->spec));
    const size_t ns = (size_t)M * Mh;
    k_sk_scale_GR<<<(unsigned)((ns + tb - 1) / tb), tb, 0, h->stream>>>(M, Mh, wd.twopi_L, wd.inv4xi2, wd.one_m_eta,
                                                                        wd.scale / h->eta, K->spec);
    FBIM_CUFFT_TRY(h, cufftExecZ2D(K->plan_i2, K->spec, K->grid));
    k_sk_interp<<<N, 128, 0, h->stream>>>(N, h->x, M, h->P, hh, wd.a, wd.g0, K->grid, 1.0, b);
    h->launches += 4;
    FBIM_CUDA_TRY(h, cudaGetLastError());
    return FBIM_OK;
}

namespace {
__global__ void k_sk_sub(long long n, const double* __restrict__ b, double* __restrict__ w) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] = b[i] - w[i];
}
}  // namespace

// restarted GMRES on A x = b (x starts at zero), CGS2 on the device
static fbim_status sk_gmres(fbim_handle_s* h, double tol, int max_iter, int& iters, double& rel) {
    SecondKind* K = h->sk;
    const int N = h->N, n = 2 * N + 3 * h->n_b, m = K->m, hs = cgs_hist_stride(m), tb = 256;
    double bn = 0;
    FBIM_TRY(dev_norm2(h, n, K->b, bn));
    FBIM_CUDA_TRY(h, cudaMemsetAsync(K->r, 0, sizeof(double) * n, h->stream));  // r holds x
    iters = 0;
    rel = 0;
    if (bn == 0) return FBIM_OK;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), yv(m);
    double* X = K->r;
    bool first = true;
    while (true) {
        double beta = 0;
        if (first) {
            FBIM_CUDA_TRY(h, cudaMemcpyAsync(K->w, K->b, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
            beta = bn;
        } else {
            FBIM_TRY(sk_apply(h, X, K->w));
            k_sk_sub<<<(n + tb - 1) / tb, tb, 0, h->stream>>>(n, K->b, K->w);
            h->launches += 1;
            FBIM_TRY(dev_norm2(h, n, K->w, beta));
        }
        first = false;
        rel = beta / bn;
        if (!std::isfinite(rel)) {
            h->fail("second-kind GMRES residual is not finite");
            return FBIM_ERR_NONFINITE;
        }
        if (rel <= tol || iters >= max_iter) return FBIM_OK;
        cgs_start(h, K->cgs, 1.0 / beta, K->w, K->V, K->vin);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int used = 0;
        for (int k = 0; k < m && iters < max_iter; ++k) {
            FBIM_TRY(sk_apply(h, K->vin, K->w));
            cgs_step(h, K->cgs, K->V, K->w, true, K->vin);
            FBIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
            const double* row = K->cgs.hist_host + (size_t)k * hs;
            double* col = &H[(size_t)k * (m + 1)];
            for (int i = 0; i <= k; ++i) col[i] = row[i] + row[(m + 1) + i];
            const double hn = std::sqrt(std::max(row[2 * (m + 1)], 0.0));
            col[k + 1] = hn;
            for (int i = 0; i < k; ++i) {
                const double t0 = cs[i] * col[i] + sn[i] * col[i + 1];
                col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
                col[i] = t0;
            }
            const double den = std::hypot(col[k], col[k + 1]);
            cs[k] = den > 0 ? col[k] / den : 1.0;
            sn[k] = den > 0 ? col[k + 1] / den : 0.0;
            col[k] = den;
            col[k + 1] = 0.0;
            g[k + 1] = -sn[k] * g[k];
            g[k] = cs[k] * g[k];
            ++iters;
            used = k + 1;
            if (!std::isfinite(g[k + 1])) {
                h->fail("second-kind GMRES iterate is not finite");
                return FBIM_ERR_NONFINITE;
            }
            if (std::fabs(g[k + 1]) <= tol * bn || hn == 0.0) break;
        }
        for (int i = used - 1; i >= 0; --i) {
            double acc = g[i];
            for (int j = i + 1; j < used; ++j) acc -= H[(size_t)j * (m + 1) + i] * yv[j];
            yv[i] = acc / H[(size_t)i * (m + 1) + i];
        }
        FBIM_CUDA_TRY(h, cudaMemcpyAsync(K->y, yv.data(), sizeof(double) * used, cudaMemcpyHostToDevice, h->stream));
        dev_combine(h, n, used, K->V, K->cgs.ld, K->y, 1.0, X);
        FBIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));  // yv outlives its copy
    }
}

fbim_status second_kind_solve(fbim_handle_s* h, const double* F, double tol, int max_iter, double* U, double* phi,
                              int* iters, double* rel_out) {
    FBIM_TRY(ensure_solver(h));
    FBIM_TRY(sk_setup(h));
    SecondKind* K = h->sk;
    const int N = h->N;
    FBIM_TRY(sk_rhs(h, F, K->b));
    int it = 0;
    double est = 0;
    FBIM_TRY(sk_gmres(h, tol, max_iter, it, est));
    // the reported residual is measured: |b - A x| / |b|
    const int n = 2 * N + 3 * h->n_b, tb = 256;
    FBIM_TRY(sk_apply(h, K->r, K->w));
    k_sk_sub<<<(n + tb - 1) / tb, tb, 0, h->stream>>>(n, K->b, K->w);
    h->launches += 1;
    double rn = 0, bn = 0;
    FBIM_TRY(dev_norm2(h, n, K->w, rn));
    FBIM_TRY(dev_norm2(h, n, K->b, bn));
    const double rel = bn > 0 ? rn / bn : 0.0;
    FBIM_CUDA_TRY(h, cudaMemcpyAsync(U, K->r + 2 * (size_t)N, sizeof(double) * 3 * h->n_b, cudaMemcpyDeviceToDevice,
                                     h->stream));
    if (phi)
        FBIM_CUDA_TRY(h, cudaMemcpyAsync(phi, K->r, sizeof(double) * 2 * (size_t)N, cudaMemcpyDeviceToDevice,
                                         h->stream));
    FBIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (iters) *iters = it;
    if (rel_out) *rel_out = rel;
    if (!std::isfinite(rel)) {
        h->fail("second-kind solve produced non-finite values");
        return FBIM_ERR_NONFINITE;
    }
    if (rel > tol) {
        h->fail("second-kind GMRES reached the iteration cap before the tolerance");
        return FBIM_ERR_NOT_CONVERGED;
    }
    return FBIM_OK;
}

}  // namespace fbim

extern "C" fbim_status fbim_second_kind_solve(fbim_handle h, const double* F_dev, double tol, int max_iter,
                                              double* U_dev, double* phi_dev, int* iters, double* rel_residual) {
    if (!h || !F_dev || !U_dev || !(tol > 0) || max_iter <= 0) return FBIM_ERR_INVALID_ARG;
    try {
        if (cudaSetDevice(h->device) != cudaSuccess) return FBIM_ERR_CUDA;
        return fbim::second_kind_solve(h, F_dev, tol, max_iter, U_dev, phi_dev, iters, rel_residual);
    } catch (...) {
        h->fail("unexpected host exception in fbim_second_kind_solve");
        return FBIM_ERR_SETUP;
    }
}

extern "C" fbim_status fbim_second_kind_apply(fbim_handle h, const double* x_dev, double* y_dev) {
    if (!h || !x_dev || !y_dev || x_dev == y_dev) return FBIM_ERR_INVALID_ARG;
    try {
        if (cudaSetDevice(h->device) != cudaSuccess) return FBIM_ERR_CUDA;
        FBIM_TRY(fbim::ensure_solver(h));
        FBIM_TRY(fbim::sk_setup(h));
        FBIM_TRY(fbim::sk_apply(h, x_dev, y_dev));
        FBIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        return FBIM_OK;
    } catch (...) {
        h->fail("unexpected host exception in fbim_second_kind_apply");
        return FBIM_ERR_SETUP;
    }
}

extern "C" fbim_status fbim_second_kind_rhs(fbim_handle h, const double* F_dev, double* b_dev) {
    if (!h || !F_dev || !b_dev) return FBIM_ERR_INVALID_ARG;
    try {
        if (cudaSetDevice(h->device) != cudaSuccess) return FBIM_ERR_CUDA;
        FBIM_TRY(fbim::ensure_solver(h));
        FBIM_TRY(fbim::sk_setup(h));
        FBIM_TRY(fbim::sk_rhs(h, F_dev, b_dev));
        FBIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        return FBIM_OK;
    } catch (...) {
        h->fail("unexpected host exception in fbim_second_kind_rhs");
        return FBIM_ERR_SETUP;
    }
}
