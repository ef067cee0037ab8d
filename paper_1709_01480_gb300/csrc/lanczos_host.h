// Host side of the Lanczos square root (Sec. 3.3): the coefficients
//     c = |w| f(T_k) e_1,  f = sqrt (negative Ritz values clipped to zero),
// of the approximation y_k = V_k c to f(A) w, from the k x k symmetric tridiagonal
// T_k = tridiag(beta, alpha, beta) the iteration builds.
//
// T_k = S diag(lambda) S^T by the symmetric tridiagonal QR algorithm with implicit
// Wilkinson shifts (Golub & Van Loan, Matrix Computations, Sec. 8.3: Wilkinson
// shift from the trailing 2 x 2, one bulge-chasing sweep of Givens rotations per
// step, deflation of negligible off-diagonals, relative to the neighbours or to
// ||T||).  T is held dense but each rotation
// only touches the band around its two rows; the rotations accumulate into S.
// O(k^3) flops with a small constant; k stays below ~50 here, and the entries of T
// are of the order of the operator's norm, so the plain sqrt(x^2 + z^2) cannot overflow.
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

namespace fbim {

// Eigen-decomposition of the k x k symmetric tridiagonal matrix (diagonal a[0..k),
// off-diagonal b[0..k-1)): lam[j] and S (row-major, eigenvectors as columns).
inline void tridiag_eig(const double* a, const double* b, int k, std::vector<double>& lam, std::vector<double>& S) {
    std::vector<double> T((size_t)k * k, 0.0);
    S.assign((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i) {
        T[(size_t)i * k + i] = a[i];
        S[(size_t)i * k + i] = 1.0;
        if (i + 1 < k) T[(size_t)i * k + i + 1] = T[(size_t)(i + 1) * k + i] = b[i];
    }
    auto at = [&](int i, int j) -> double& { return T[(size_t)i * k + j]; };
    // G = I except the (p, p+1) block [c s; -s c]; T <- G^T T G on the band, S <- S G
    auto rotate = [&](int p, double c, double s, int lo, int hi) {
        const int q = p + 1, j0 = std::max(lo, p - 1), j1 = std::min(hi, q + 1);
        for (int j = j0; j <= j1; ++j) {
            const double tp = at(p, j), tq = at(q, j);
            at(p, j) = c * tp - s * tq;
            at(q, j) = s * tp + c * tq;
        }
        for (int i = j0; i <= j1; ++i) {
            const double tp = at(i, p), tq = at(i, q);
            at(i, p) = c * tp - s * tq;
            at(i, q) = s * tp + c * tq;
        }
        for (int i = 0; i < k; ++i) {
            double& sp = S[(size_t)i * k + p];
            double& sq = S[(size_t)i * k + q];
            const double tp = sp, tq = sq;
            sp = c * tp - s * tq;
            sq = s * tp + c * tq;
        }
    };
    const double eps = 2.220446049250313e-16;
    // An off-diagonal is negligible below eps times its two diagonal neighbours, or below
    // eps ||T||: a cluster of (numerically) zero eigenvalues would otherwise never deflate,
    // its neighbours being zero too.
    double tnorm = 0.0;
    for (int i = 0; i < k; ++i)
        tnorm = std::max(tnorm, std::fabs(a[i]) + (i > 0 ? std::fabs(b[i - 1]) : 0.0) +
                                    (i + 1 < k ? std::fabs(b[i]) : 0.0));
    auto negligible = [&](int i) {  // the off-diagonal between rows i - 1 and i
        const double e = std::fabs(at(i, i - 1));
        return e <= eps * (std::fabs(at(i, i)) + std::fabs(at(i - 1, i - 1))) || e <= eps * tnorm;
    };
    int hi = k - 1, guard = 0;
    while (hi > 0 && guard < 60 * k) {
        // deflate a negligible off-diagonal at the bottom
        if (negligible(hi)) {
            at(hi, hi - 1) = at(hi - 1, hi) = 0.0;
            --hi;
            continue;
        }
        // the unreduced block [lo, hi]
        int lo = hi - 1;
        while (lo > 0 && !negligible(lo)) --lo;
        if (lo > 0) at(lo, lo - 1) = at(lo - 1, lo) = 0.0;
        // Wilkinson shift: the eigenvalue of the trailing 2 x 2 closer to its last entry
        const double d = 0.5 * (at(hi - 1, hi - 1) - at(hi, hi)), e = at(hi, hi - 1);
        const double den = d + (d >= 0 ? 1.0 : -1.0) * std::sqrt(d * d + e * e);
        const double mu = den != 0.0 ? at(hi, hi) - e * e / den : at(hi, hi) - std::fabs(e);
        // implicit step: the first rotation from the shifted first column, then chase the bulge
        double x = at(lo, lo) - mu, z = at(lo + 1, lo);
        for (int p = lo; p < hi; ++p) {
            const double r = std::sqrt(x * x + z * z);
            const double c = r > 0 ? x / r : 1.0, s = r > 0 ? -z / r : 0.0;
            rotate(p, c, s, lo, hi);
            if (p + 2 <= hi) {
                x = at(p + 1, p);
                z = at(p + 2, p);
            }
        }
        ++guard;
    }
    lam.resize(k);
    for (int i = 0; i < k; ++i) lam[i] = at(i, i);
}

// c = wnorm sqrt(T_k) e_1 (length k); negative Ritz values clipped to zero.
inline std::vector<double> lanczos_sqrt_coeffs(const double* alpha, const double* beta, int k, double wnorm) {
    std::vector<double> lam, S;
    tridiag_eig(alpha, beta, k, lam, S);
    std::vector<double> c(k, 0.0);
    for (int j = 0; j < k; ++j) {
        const double f = lam[j] > 0 ? std::sqrt(lam[j]) : 0.0;
        const double w = f * S[j];  // S[0][j] = e_1^T s_j
        if (w == 0.0) continue;
        for (int i = 0; i < k; ++i) c[i] += S[(size_t)i * k + j] * w;
    }
    for (auto& v : c) v *= wnorm;
    return c;
}

}  // namespace fbim
