// Host-side setup of the FBIM library: Ewald parameter rules (Sec. 3.2), the
// exponential integral E1 (Sec. 3.2, Eq. expint), the log-singular end
// correction (Sec. 3.1, Alpert's hybrid Gauss-trapezoidal rule) and the
// reference body's correction band M(a)_ref (Sec. 3.2).
//
// Everything here runs once per handle, in long double where the derivation
// needs it, and feeds constant tables to the device kernels.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "fbim_internal.h"

namespace fbim {

namespace {
thread_local std::string g_error;
using ld = long double;
const ld kPi = 3.141592653589793238462643383279502884L;
const ld kEulerGamma = 0.577215664901532860606512090082402431L;
}  // namespace

void set_global_error(const std::string& msg) { g_error = msg; }
const char* global_error() { return g_error.c_str(); }

// ---------------------------------------------------------------------------
// E1(z), z > 0: power series E1 = -gamma - ln z - sum_k (-z)^k / (k k!) for
// z < 3; for z >= 3 the continued fraction e^{-z} / (z + 1 - 1/(z + 3 - 4/(z + 5 - ...)))
// evaluated bottom-up at a fixed depth.  Both are textbook expansions of the
// exponential integral (Abramowitz & Stegun 5.1.11 and 5.1.22).
// ---------------------------------------------------------------------------
static ld e1_ld(ld z) {
    if (!(z > 0)) return INFINITY;
    if (z < 3) {
        ld term = 1, sum = 0;
        for (int k = 1; k <= 80; ++k) {
            term *= -z / k;
            ld add = term / k;
            sum += add;
            if (fabsl(add) < 1e-24L * fabsl(sum)) break;
        }
        return -kEulerGamma - logl(z) - sum;
    }
    const int depth = 80;
    ld f = z + (2 * depth + 1);
    for (int k = depth; k >= 1; --k) f = z + (2 * k - 1) - (ld)k * k / f;
    return expl(-z) / f;
}

double host_e1(double zd) { return (double)e1_ld(zd); }

// Chebyshev interpolant of S(z) = (E1(z) + ln z)/2 - e^{-z} on [0, zmax] at the
// deg + 1 Chebyshev points of the first kind.  S is entire (E1(z) + ln z =
// -gamma + sum_k (-1)^{k+1} z^k/(k k!)), so the coefficients decay fast: degree
// 28 reaches 1e-9 and degree 44 reaches 1e-14 on [0, 36].
void e1_chebyshev(double zmax, int deg, std::vector<double>& coef) {
    const int n = deg + 1;
    std::vector<ld> f(n);
    for (int k = 0; k < n; ++k) {
        ld th = kPi * (k + 0.5L) / n;
        ld z = 0.5L * zmax * (cosl(th) + 1);
        ld S;
        if (z < 1e-6L) {
            S = 0.5L * (-kEulerGamma + z - z * z / 4) - expl(-z);
        } else {
            S = 0.5L * (e1_ld(z) + logl(z)) - expl(-z);
        }
        f[k] = S;
    }
    coef.assign(n, 0.0);
    for (int j = 0; j < n; ++j) {
        ld acc = 0;
        for (int k = 0; k < n; ++k) acc += f[k] * cosl(j * kPi * (k + 0.5L) / n);
        coef[j] = (double)(acc * 2 / n);
    }
    coef[0] *= 0.5;
}

// S(z) = (E1(z) + ln z)/2 - e^{-z} in long double: the power series of its entire
// part for z < 3 (no logarithm to cancel; also valid for z < 0), E1 by its continued
// fraction above.
static ld s_ld(ld z) {
    if (z < 3) {
        ld term = 1, sum = 0;
        for (int k = 1; k <= 80; ++k) {
            term *= -z / k;
            const ld add = term / k;
            sum += add;
            if (fabsl(add) <= 1e-24L * fabsl(sum)) break;
        }
        return 0.5L * (-kEulerGamma - sum) - expl(-z);
    }
    return 0.5L * (e1_ld(z) + logl(z)) - expl(-z);
}

void e1_piecewise(double zmax, int K, int D, std::vector<float>& zc, float& inv_w, std::vector<double>& cS,
                  std::vector<double>& cE) {
    const ld w = (ld)zmax / (2 * K);
    inv_w = (float)(1.0L / w);
    const ld hw = 1.0L / (ld)inv_w;  // the half-width the device's t = (z - z_c) inv_w implies
    const int n = D + 1;
    zc.assign(K, 0.f);
    cS.assign((size_t)K * n, 0.0);
    cE.assign((size_t)K * n, 0.0);
    // monomial coefficients of T_0 .. T_D: T[m][j] = coefficient of t^j in T_m(t)
    std::vector<ld> T((size_t)n * n, 0.0L);
    T[0] = 1;
    if (n > 1) T[(size_t)1 * n + 1] = 1;
    for (int m = 2; m < n; ++m)
        for (int j = 0; j < n; ++j)
            T[(size_t)m * n + j] = (j > 0 ? 2 * T[(size_t)(m - 1) * n + j - 1] : 0) - T[(size_t)(m - 2) * n + j];
    const ld margin = 1.05L;  // t may pass +-1 by the rounding of z_c, inv_w and the piece index
    std::vector<ld> f(n), a(n);
    for (int k = 0; k < K; ++k) {
        zc[k] = (float)((2 * k + 1) * w);
        const ld c = zc[k];
        for (int i = 0; i < n; ++i) {
            const ld t = margin * cosl(kPi * (i + 0.5L) / n);
            f[i] = s_ld(c + hw * t);  // the first piece's points reach below 0: S is entire
        }
        for (int j = 0; j < n; ++j) {
            ld acc = 0;
            for (int i = 0; i < n; ++i) acc += f[i] * cosl(j * kPi * (i + 0.5L) / n);
            a[j] = acc * 2 / n;
        }
        a[0] *= 0.5L;
        // p(t) = sum_m a_m T_m(t / margin)
        ld scale = 1;
        for (int j = 0; j < n; ++j) {
            ld acc = 0;
            for (int m = j; m < n; ++m) acc += a[m] * T[(size_t)m * n + j];
            cS[(size_t)k * n + j] = (double)(acc * scale);
            scale /= margin;
        }
        // e^{-(c + hw t)} = e^{-c} sum_j (-hw)^j t^j / j!
        ld term = expl(-c);
        for (int j = 0; j < n; ++j) {
            cE[(size_t)k * n + j] = (double)term;
            term *= -hw / (j + 1);
        }
    }
}

// ---------------------------------------------------------------------------
// Parameter rules (Sec. 3.2): C_r e^{-xi^2 r_c^2} <= tol, C_w H^(k_max) <= tol,
// e^{-pi P / 2} <= tol, m = sqrt(pi P), eta_s = (2 w xi / m)^2 with w = P h / 2.
// ---------------------------------------------------------------------------
static bool nice_size(int n) {
    for (int p : {2, 3, 5, 7})
        while (n % p == 0) n /= p;
    return n == 1;
}

static int next_nice_even(int n) {
    if (n < 8) n = 8;
    if (n % 2) ++n;
    while (!nice_size(n)) n += 2;
    return n;
}

fbim_status choose_ewald(double L, double r_c, double tol, double xi_in, int& n_box, double& r_c_out,
                         double& xi, int& M, int& P, double& eta_s, std::string& err) {
    if (!(L > 0) || !(tol > 0 && tol < 1) || !(r_c > 0)) {
        err = "choose_ewald: need L > 0, 0 < tol < 1 and r_c > 0";
        return FBIM_ERR_INVALID_ARG;
    }
    const double C_r = 100.0, C_w = 1.0;
    n_box = (int)std::floor(L / r_c * (1.0 + 1e-12));
    if (n_box < 3) {
        err = "choose_ewald: r_c must be at most L/3 (nine distinct neighbour cells)";
        return FBIM_ERR_INVALID_ARG;
    }
    r_c_out = L / n_box;
    xi = xi_in > 0 ? xi_in : std::sqrt(std::log(C_r / tol)) / r_c_out;
    // Wave space: the first dropped mode must satisfy C_w H^(k_max) <= tol, where the
    // Hasimoto factor H^ = (1 + q) e^{-q}, q = k^2/4xi^2, carries the polynomial
    // prefactor that a bare C_w e^{-q} bound leaves out.  Solve q = ln(C_w/tol) + ln(1 + q).
    double q = std::log(C_w / tol);
    for (int it = 0; it < 50; ++it) q = std::log(C_w / tol) + std::log1p(q);
    double kmax = 2.0 * xi * std::sqrt(q);
    M = next_nice_even((int)std::ceil(kmax * L / M_PI));
    P = (int)std::ceil(2.0 * std::log(1.0 / tol) / M_PI);
    if (P % 2 == 0) ++P;
    for (int guard = 0; guard < 200; ++guard) {
        double h = L / M;
        double w = P * h / 2.0;
        double m = std::sqrt(M_PI * P);
        eta_s = std::pow(2.0 * w * xi / m, 2);
        if (eta_s < 1.0 && P <= M) return FBIM_OK;
        M = next_nice_even(M + 2);
    }
    err = "choose_ewald: could not reach eta_s < 1";
    return FBIM_ERR_SETUP;
}

// ---------------------------------------------------------------------------
// Log-singular end correction.  On each side of the target the trapezoidal
// nodes at offsets 1..a-1 are replaced by j auxiliary nodes v_k (units of the
// spacing) with weights w_k, chosen so that the rule integrates x^p and
// x^p log x exactly for p = 0..j-1.  With the generalised Euler-Maclaurin
// (zeta-function) expansion of h sum_{i>=1} f(ih) these conditions read
//     sum_k w_k v_k^p         = sum_{i<a} i^p - zeta(-p)
//     sum_k w_k v_k^p ln v_k  = sum_{i<a} i^p ln i + zeta'(-p).
// Order = j + 1; order 4 uses (j, a) = (3, 3), order 8 uses (7, 5).
// ---------------------------------------------------------------------------
namespace {

// Bernoulli numbers B_{2k} from zeta(2k) = sum n^{-2k}:  B_{2k} = (-1)^{k+1} 2 (2k)! zeta(2k) / (2 pi)^{2k}.
ld bernoulli_even(int k) {
    ld z;
    if (k == 1) {
        z = kPi * kPi / 6;
    } else {
        const int Nt = 2000;
        z = 0;
        for (int n = Nt - 1; n >= 1; --n) z += powl((ld)n, (ld)(-2 * k));
        ld s = 2 * k;
        // Euler-Maclaurin tail sum_{n >= Nt} n^{-s}
        z += powl((ld)Nt, 1 - s) / (s - 1) + 0.5L * powl((ld)Nt, -s) + s / 12.0L * powl((ld)Nt, -s - 1);
    }
    ld fact = 1;
    for (int i = 2; i <= 2 * k; ++i) fact *= i;
    ld b = 2 * fact * z / powl(2 * kPi, 2 * k);
    return (k % 2 == 1) ? b : -b;
}

ld zeta_neg(int p) {  // zeta(-p) = (-1)^p B_{p+1}/(p+1)
    if (p == 0) return -0.5L;
    if (p % 2 == 0) return 0;
    int k = (p + 1) / 2;
    return -bernoulli_even(k) / (p + 1);
}

// Sums over k >= 1 of k^{-s} and of ln(k) k^{-s} (s >= 2): direct sum to N - 1 plus
// the Euler-Maclaurin tail  int_N^inf f + f(N)/2 - f'(N)/12.
ld zeta_pos(ld s) {
    const int N = 4000;
    ld acc = 0;
    for (int k = N - 1; k >= 1; --k) acc += powl((ld)k, -s);
    ld fN = powl((ld)N, -s);
    return acc + N * fN / (s - 1) + fN / 2 + s * fN / (12.0L * N);
}
ld zeta_prime_pos(ld s) {  // zeta'(s) = -sum ln k k^{-s}
    const int N = 4000;
    ld acc = 0;
    for (int k = N - 1; k >= 2; --k) acc += logl((ld)k) * powl((ld)k, -s);
    ld lnN = logl((ld)N), fN = powl((ld)N, -s);
    ld integral = N * fN * (lnN / (s - 1) + 1 / ((s - 1) * (s - 1)));
    ld dfN = fN / N * (1 - s * lnN);
    return -(acc + integral + lnN * fN / 2 - dfN / 12);
}

// zeta'(-p) from the functional equation, which avoids the cancellation of a
// direct continuation:
//   p = 0:          zeta'(0) = -ln(2 pi) / 2
//   p = 2n:         zeta'(-2n) = (-1)^n (2n)! zeta(2n+1) / (2 (2 pi)^{2n})
//   p = 2n - 1:     zeta'(1-2n) = zeta(1-2n) [ln(2 pi) - psi(2n) - zeta'(2n)/zeta(2n)],
//                   psi(2n) = -gamma + sum_{k<2n} 1/k.
ld zeta_prime_neg(int p) {
    if (p == 0) return -0.5L * logl(2 * kPi);
    if (p % 2 == 0) {
        int n = p / 2;
        ld fact = 1;
        for (int i = 2; i <= 2 * n; ++i) fact *= i;
        ld sgn = (n % 2) ? -1 : 1;
        return sgn * fact * zeta_pos(2 * n + 1) / (2 * powl(2 * kPi, 2 * n));
    }
    int n = (p + 1) / 2;
    ld psi = -kEulerGamma;
    for (int k = 1; k < 2 * n; ++k) psi += 1.0L / k;
    ld z2n = zeta_pos(2 * n);
    return zeta_neg(p) * (logl(2 * kPi) - psi - zeta_prime_pos(2 * n) / z2n);
}

bool solve_dense(std::vector<ld>& A, std::vector<ld>& b, int n) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabsl(A[r * n + c]) > fabsl(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0) return false;
        if (piv != c) {
            for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
            std::swap(b[c], b[piv]);
        }
        for (int r = c + 1; r < n; ++r) {
            ld f = A[r * n + c] / A[c * n + c];
            for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        ld acc = b[r];
        for (int k = r + 1; k < n; ++k) acc -= A[r * n + k] * b[k];
        b[r] = acc / A[r * n + r];
    }
    return true;
}

ld rule_residual(const std::vector<ld>& z, int j, const std::vector<ld>& m, const std::vector<ld>& nn,
                 std::vector<ld>* r, std::vector<ld>* J) {
    ld norm = 0;
    for (int p = 0; p < j; ++p) {
        ld r1 = -m[p], r2 = -nn[p];
        for (int k = 0; k < j; ++k) {
            ld v = z[k], w = z[j + k], lv = logl(v);
            ld vp = powl(v, (ld)p);
            ld dvp = p > 0 ? p * powl(v, (ld)(p - 1)) : 0;
            r1 += w * vp;
            r2 += w * vp * lv;
            if (J) {
                (*J)[p * 2 * j + k] = w * dvp;
                (*J)[p * 2 * j + j + k] = vp;
                (*J)[(j + p) * 2 * j + k] = w * (dvp * lv + vp / v);
                (*J)[(j + p) * 2 * j + j + k] = vp * lv;
            }
        }
        if (r) {
            (*r)[p] = r1;
            (*r)[j + p] = r2;
        }
        norm += r1 * r1 + r2 * r2;
    }
    return sqrtl(norm);
}

}  // namespace

fbim_status alpert_rule(int order, std::vector<double>& vout, std::vector<double>& wout, int& a, std::string& err) {
    int j;
    if (order == 4) {
        j = 3;
        a = 3;
    } else if (order == 8) {
        j = 7;
        a = 5;
    } else {
        err = "alpert_order must be 4 or 8";
        return FBIM_ERR_INVALID_ARG;
    }
    std::vector<ld> m(j), nn(j);
    for (int p = 0; p < j; ++p) {
        ld sm = 0, sl = 0;
        for (int i = 1; i < a; ++i) {
            sm += powl((ld)i, (ld)p);
            sl += powl((ld)i, (ld)p) * logl((ld)i);
        }
        m[p] = sm - zeta_neg(p);
        nn[p] = sl + zeta_prime_neg(p);
    }
    const int n = 2 * j;
    const double shapes[] = {2.0, 1.5, 2.5, 3.0, 1.2, 4.0};
    const double scales[] = {1.0, 0.8, 1.2, 0.6};
    for (double shp : shapes) {
        for (double scl : scales) {
            std::vector<ld> z(n), r(n), J(n * n);
            for (int k = 0; k < j; ++k) {
                z[k] = scl * a * powl((k + 0.5L) / j, (ld)shp);
                z[j + k] = (a - 0.5L) / j;
            }
            ld res = rule_residual(z, j, m, nn, &r, &J);
            for (int it = 0; it < 300 && res > 1e-17L; ++it) {
                std::vector<ld> dz(r);
                for (auto& t : dz) t = -t;
                std::vector<ld> Jc(J);
                if (!solve_dense(Jc, dz, n)) break;
                ld lam = 1;
                std::vector<ld> zn(n);
                ld rn = res;
                while (lam > 1e-6L) {
                    bool pos = true;
                    for (int k = 0; k < n; ++k) zn[k] = z[k] + lam * dz[k];
                    for (int k = 0; k < j; ++k) pos = pos && zn[k] > 0;
                    if (pos) {
                        rn = rule_residual(zn, j, m, nn, nullptr, nullptr);
                        if (rn < res || lam < 1e-3L) break;
                    }
                    lam *= 0.5L;
                }
                z = zn;
                res = rule_residual(z, j, m, nn, &r, &J);
            }
            bool ok = res < 1e-15L;
            for (int k = 0; k < j; ++k) ok = ok && z[k] > 0 && z[k] < a + 1 && z[j + k] > 0;
            if (!ok) continue;
            std::vector<int> idx(j);
            for (int k = 0; k < j; ++k) idx[k] = k;
            for (int x1 = 0; x1 < j; ++x1)
                for (int x2 = x1 + 1; x2 < j; ++x2)
                    if (z[idx[x2]] < z[idx[x1]]) std::swap(idx[x1], idx[x2]);
            vout.resize(j);
            wout.resize(j);
            for (int k = 0; k < j; ++k) {
                vout[k] = (double)z[idx[k]];
                wout[k] = (double)z[j + idx[k]];
            }
            return FBIM_OK;
        }
    }
    err = "alpert_rule: Newton iteration found no admissible rule";
    return FBIM_ERR_SETUP;
}

// ---------------------------------------------------------------------------
// Reference band M(a)_ref (Sec. 3.2): for target i of the reference body,
//   (M(a) mu)_i = - sum_{0<|o|<a} G^(r)(x_i - x_{i+o}) mu_{i+o}
//                 + sum_{k, +-} w_k G^(r)(x_i - gamma(s_i +- v_k Ds)) sum_o l_o^{k,+-} mu_{i+o}
// where gamma between nodes is the trigonometric interpolant of the nodes and
// l are Lagrange weights over the order+2 nodes nearest to the auxiliary point.
// Stored symmetrised, (M(a) + M(a)^T)/2, as [n_p][2 band + 1][2][2].
// ---------------------------------------------------------------------------
void g_real_host(double rx, double ry, double xi, double eta, double G[4]) {
    double r2 = rx * rx + ry * ry;
    double z = xi * xi * r2;
    double e = std::exp(-z);
    double a = 0.5 * host_e1(z) - e;
    double b = e / r2;
    double c = 1.0 / (4.0 * M_PI * eta);
    G[0] = c * (a + b * rx * rx);
    G[1] = c * (b * rx * ry);
    G[2] = G[1];
    G[3] = c * (a + b * ry * ry);
}

namespace {

struct TrigCurve {
    int n;
    std::vector<double> cr, ci;  // [n][2] Fourier coefficients (real, imaginary), k = 0..n-1
    explicit TrigCurve(const std::vector<double>& nodes) : n((int)nodes.size() / 2), cr(nodes.size()), ci(nodes.size()) {
        for (int k = 0; k < n; ++k)
            for (int c = 0; c < 2; ++c) {
                double sr = 0, si = 0;
                for (int jj = 0; jj < n; ++jj) {
                    double ang = -2.0 * M_PI * (double)k * jj / n;
                    sr += nodes[2 * jj + c] * std::cos(ang);
                    si += nodes[2 * jj + c] * std::sin(ang);
                }
                cr[2 * k + c] = sr / n;
                ci[2 * k + c] = si / n;
            }
    }
    // gamma(s): symmetric interpolant, Nyquist term carried by cos(n/2 s)
    void eval(double s, double out[2]) const {
        for (int c = 0; c < 2; ++c) {
            double acc = cr[c];
            for (int k = 1; k < n; ++k) {
                int kk = k <= n / 2 ? k : k - n;
                if (n % 2 == 0 && k == n / 2) {
                    acc += cr[2 * k + c] * std::cos(kk * s);
                    continue;
                }
                acc += cr[2 * k + c] * std::cos(kk * s) - ci[2 * k + c] * std::sin(kk * s);
            }
            out[c] = acc;
        }
    }
};

void lagrange(double t, int q, std::vector<int>& offs, std::vector<double>& wts) {
    int base = (int)std::floor(t);
    offs.resize(q);
    wts.assign(q, 1.0);
    for (int i = 0; i < q; ++i) offs[i] = base - q / 2 + 1 + i;
    for (int i = 0; i < q; ++i)
        for (int k = 0; k < q; ++k)
            if (k != i) wts[i] *= (t - offs[k]) / (double)(offs[i] - offs[k]);
}

}  // namespace

fbim_status alpert_reference_band(fbim_handle_s* h, std::vector<double>& band_out) {
    std::vector<double> v, w;
    int a;
    std::string err;
    fbim_status st = alpert_rule(h->order, v, w, a, err);
    if (st != FBIM_OK) {
        h->fail(err);
        return st;
    }
    const int n = h->n_p, q = h->order + 2;
    const int j = (int)v.size();
    int band = a - 1;
    for (int k = 0; k < j; ++k) band = std::max(band, (int)std::floor(v[k]) + q / 2);
    if (2 * band + 1 > n) {
        h->fail("n_p too small for the Alpert band");
        return FBIM_ERR_INVALID_ARG;
    }
    h->aj = j;
    h->aa = a;
    h->band = band;
    const int B = 2 * band + 1;
    std::vector<double> A((size_t)n * B * 4, 0.0);  // [i][o + band][2][2], not symmetrised
    TrigCurve curve(h->host_ref);
    const double ds = 2.0 * M_PI / n;
    const double* X = h->host_ref.data();
    for (int i = 0; i < n; ++i) {
        double G[4];
        for (int o = 1; o < a; ++o)
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                int nb = ((i + sgn * o) % n + n) % n;
                g_real_host(X[2 * i] - X[2 * nb], X[2 * i + 1] - X[2 * nb + 1], h->xi, h->eta, G);
                double* dst = &A[((size_t)i * B + (sgn * o + band)) * 4];
                for (int t = 0; t < 4; ++t) dst[t] -= G[t];
            }
        for (int k = 0; k < j; ++k)
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                double t = sgn * v[k];
                double y[2];
                curve.eval((i + t) * ds, y);
                g_real_host(X[2 * i] - y[0], X[2 * i + 1] - y[1], h->xi, h->eta, G);
                std::vector<int> offs;
                std::vector<double> lw;
                lagrange(t, q, offs, lw);
                for (int u = 0; u < q; ++u) {
                    double* dst = &A[((size_t)i * B + (offs[u] + band)) * 4];
                    for (int tt = 0; tt < 4; ++tt) dst[tt] += w[k] * lw[u] * G[tt];
                }
            }
    }
    // symmetrise: S[i][o] = (A[i][o] + A[i+o][-o]^T) / 2
    band_out.assign(A.size(), 0.0);
    for (int i = 0; i < n; ++i)
        for (int o = -band; o <= band; ++o) {
            int nb = ((i + o) % n + n) % n;
            const double* a1 = &A[((size_t)i * B + (o + band)) * 4];
            const double* a2 = &A[((size_t)nb * B + (-o + band)) * 4];
            double* d = &band_out[((size_t)i * B + (o + band)) * 4];
            d[0] = 0.5 * (a1[0] + a2[0]);
            d[1] = 0.5 * (a1[1] + a2[2]);
            d[2] = 0.5 * (a1[2] + a2[1]);
            d[3] = 0.5 * (a1[3] + a2[3]);
        }
    return FBIM_OK;
}

// ---------------------------------------------------------------------------
// Dense reference blocks for the preconditioners (Sec. 3.4): the reference body
// alone in the periodic box.
//   M(r)_ref = M(t)_ref + M(a)_ref,sym      (real space, used by the Lanczos G_ref)
//   M_ref    = M(r)_ref + M(w)_ref          (used by the GMRES block preconditioner)
// M(w)_ref[m][n] = G^(w)_xi(x_m - x_n) is evaluated through the periodic Stokeslet,
// which the Hasimoto split reproduces for any splitting parameter: with a second,
// small xi' (real space over a few images, a few hundred Fourier modes),
//   G^(w)_xi(r) = sum_p G^(r)_xi'(r + pL) + G^(w)_xi'(r) - sum_p G^(r)_xi(r + pL),
// and at r = 0 the log singularities cancel to (1/4 pi eta) ln(xi/xi') I.
// Row-major [2 n_p][2 n_p], index 2 m + c.
// ---------------------------------------------------------------------------
void reference_blocks(fbim_handle_s* h, const std::vector<double>& band_sym, std::vector<double>& Mr,
                      std::vector<double>& Mfull) {
    const int n = h->n_p, n2 = 2 * n;
    const double L = h->L, xi = h->xi, eta = h->eta;
    const double* X = h->host_ref.data();
    Mr.assign((size_t)n2 * n2, 0.0);
    Mfull.assign((size_t)n2 * n2, 0.0);
    auto add = [&](std::vector<double>& A, int m, int k, const double G[4], double s) {
        A[(size_t)(2 * m) * n2 + 2 * k] += s * G[0];
        A[(size_t)(2 * m) * n2 + 2 * k + 1] += s * G[1];
        A[(size_t)(2 * m + 1) * n2 + 2 * k] += s * G[2];
        A[(size_t)(2 * m + 1) * n2 + 2 * k + 1] += s * G[3];
    };
    const double cut = 8.0 / xi, cut2 = cut * cut;
    // M(t)_ref: G^(r)_xi over the periodic images, m != n (the p = 0 self term excluded)
    for (int m = 0; m < n; ++m)
        for (int k = 0; k < n; ++k) {
            const int ni = (int)std::ceil(cut / L) + 1;
            for (int px = -ni; px <= ni; ++px)
                for (int py = -ni; py <= ni; ++py) {
                    if (m == k && px == 0 && py == 0) continue;
                    double rx = X[2 * m] - X[2 * k] + px * L, ry = X[2 * m + 1] - X[2 * k + 1] + py * L;
                    double r2 = rx * rx + ry * ry;
                    if (r2 >= cut2 || r2 == 0) continue;
                    double G[4];
                    g_real_host(rx, ry, xi, eta, G);
                    add(Mr, m, k, G, 1.0);
                }
        }
    // + M(a)_ref (symmetrised band)
    const int B = 2 * h->band + 1;
    for (int m = 0; m < n; ++m)
        for (int o = -h->band; o <= h->band; ++o) {
            int k = ((m + o) % n + n) % n;
            const double* a = &band_sym[((size_t)m * B + (o + h->band)) * 4];
            add(Mr, m, k, a, 1.0);
        }
    Mfull = Mr;
    // M(w)_ref through the small-xi' Ewald sum
    const double xp = 6.0 / L;
    const double cutp = 8.0 / xp;
    const int nip = (int)std::ceil(cutp / L) + 1;
    const double kcut = 2.0 * xp * std::sqrt(40.0);
    const int kmax = (int)std::ceil(kcut * L / (2.0 * M_PI));
    struct Mode { double kx, ky, w; };
    std::vector<Mode> modes;
    for (int a = -kmax; a <= kmax; ++a)
        for (int b = -kmax; b <= kmax; ++b) {
            if (a == 0 && b == 0) continue;
            double kx = 2.0 * M_PI * a / L, ky = 2.0 * M_PI * b / L, k2 = kx * kx + ky * ky;
            if (k2 > kcut * kcut) continue;
            double q = k2 / (4.0 * xp * xp);
            modes.push_back({kx, ky, (1.0 + q) * std::exp(-q) / k2 / (eta * L * L)});
        }
    for (int m = 0; m < n; ++m)
        for (int k = m; k < n; ++k) {
            double rx0 = X[2 * m] - X[2 * k], ry0 = X[2 * m + 1] - X[2 * k + 1];
            double G[4] = {0, 0, 0, 0};
            for (const Mode& md : modes) {
                double c = std::cos(md.kx * rx0 + md.ky * ry0) * md.w;
                double k2 = md.kx * md.kx + md.ky * md.ky;
                G[0] += c * (1.0 - md.kx * md.kx / k2);
                G[1] -= c * md.kx * md.ky / k2;
                G[3] += c * (1.0 - md.ky * md.ky / k2);
            }
            G[2] = G[1];
            for (int px = -nip; px <= nip; ++px)
                for (int py = -nip; py <= nip; ++py) {
                    double rx = rx0 + px * L, ry = ry0 + py * L;
                    double r2 = rx * rx + ry * ry;
                    if (r2 == 0) continue;
                    double Gp[4], Gx[4];
                    if (r2 < cutp * cutp) {
                        g_real_host(rx, ry, xp, eta, Gp);
                        for (int t = 0; t < 4; ++t) G[t] += Gp[t];
                    }
                    if (r2 < cut2) {
                        g_real_host(rx, ry, xi, eta, Gx);
                        for (int t = 0; t < 4; ++t) G[t] -= Gx[t];
                    }
                }
            if (m == k) {
                double d = std::log(xi / xp) / (4.0 * M_PI * eta);
                G[0] += d;
                G[3] += d;
            }
            add(Mfull, m, k, G, 1.0);
            if (k != m) {
                double Gt[4] = {G[0], G[2], G[1], G[3]};
                add(Mfull, k, m, Gt, 1.0);
            }
        }
}

}  // namespace fbim

extern "C" double fbim_host_expint_e1(double z) { return fbim::host_e1(z); }

extern "C" fbim_status fbim_host_alpert_rule(int order, double* v, double* w, int* a) {
    if (!v || !w || !a) return FBIM_ERR_INVALID_ARG;
    std::vector<double> vv, ww;
    std::string err;
    int aa;
    fbim_status st = fbim::alpert_rule(order, vv, ww, aa, err);
    if (st != FBIM_OK) {
        fbim::set_global_error(err);
        return st;
    }
    for (size_t k = 0; k < vv.size(); ++k) {
        v[k] = vv[k];
        w[k] = ww[k];
    }
    *a = aa;
    return FBIM_OK;
}

extern "C" fbim_status fbim_choose_ewald(double L, double r_c, double tol, double xi_in, int* n_box,
                                         double* r_c_out, double* xi, int* grid, int* support, double* eta_s) {
    int nb, M, P;
    double rc, x, es;
    std::string err;
    fbim_status st = fbim::choose_ewald(L, r_c, tol, xi_in, nb, rc, x, M, P, es, err);
    if (st != FBIM_OK) {
        fbim::set_global_error(err);
        return st;
    }
    if (n_box) *n_box = nb;
    if (r_c_out) *r_c_out = rc;
    if (xi) *xi = x;
    if (grid) *grid = M;
    if (support) *support = P;
    if (eta_s) *eta_s = es;
    return FBIM_OK;
}
