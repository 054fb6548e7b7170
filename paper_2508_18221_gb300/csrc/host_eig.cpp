// Real Schur decomposition of a small dense matrix with a real spectrum (host, FP64).
//
// Used by the XCTS solve: the angular part of the flat Laplacian of one phi mode, discretised
// on the Fourier theta nodes, is a real N_theta x N_theta matrix with real eigenvalues (a
// discrete associated-Legendre operator).  Its eigenvectors can be nearly parallel (at 6 and
// 20 theta nodes the odd modes' operator has a repeated eigenvalue), so the solve uses the
// orthogonal Schur form A = Q T Q^T instead of an eigendecomposition: Q is orthogonal at any
// spectrum, T upper triangular with the eigenvalues on its diagonal.  Steps:
//   1. Householder reduction to upper Hessenberg form, accumulating the reflections in Q;
//   2. QR iteration on the Hessenberg matrix with a Wilkinson shift from the trailing 2 x 2
//      block (an exceptional shift every tenth sweep without deflation), each Givens
//      rotation applied to the whole matrix and accumulated in Q; a subdiagonal entry below
//      the unit roundoff times its neighbours on the diagonal deflates;
//   3. a trailing 2 x 2 window keeps iterating (the shift converges to one of its real
//      eigenvalues, and the window deflates); a defective double eigenvalue, where the
//      window's subdiagonal stalls near the unit roundoff, is deflated after 40 sweeps; a
//      complex pair returns false.
// The residual max |Q T Q^T - A| / max |A| is returned; above 1e-11 the call returns false.
#include <cmath>
#include <vector>

#include "host_ops.h"

namespace gk {

namespace {

struct Mat {
    int n;
    std::vector<double> a;
    double& operator()(int i, int j) { return a[(size_t)i * n + j]; }
};

// rows k, k+1 of H (columns c0..n-1) <- G rows; columns k, k+1 of H (rows 0..r1) and of Q
// <- G^T columns, G = [[c, s], [-s, c]]
void rotate(Mat& H, Mat& Q, int k, double c, double s, int c0, int r1) {
    const int n = H.n;
    for (int j = c0; j < n; j++) {
        const double t1 = H(k, j), t2 = H(k + 1, j);
        H(k, j) = c * t1 + s * t2;
        H(k + 1, j) = -s * t1 + c * t2;
    }
    for (int i = 0; i <= r1; i++) {
        const double t1 = H(i, k), t2 = H(i, k + 1);
        H(i, k) = c * t1 + s * t2;
        H(i, k + 1) = -s * t1 + c * t2;
    }
    for (int i = 0; i < n; i++) {
        const double t1 = Q(i, k), t2 = Q(i, k + 1);
        Q(i, k) = c * t1 + s * t2;
        Q(i, k + 1) = -s * t1 + c * t2;
    }
}

void hessenberg(Mat& H, Mat& Q) {
    const int n = H.n;
    std::vector<double> v(n);
    for (int k = 0; k + 2 < n; k++) {
        double nrm = 0.0;
        for (int i = k + 1; i < n; i++) nrm += H(i, k) * H(i, k);
        nrm = std::sqrt(nrm);
        if (nrm == 0.0) continue;
        const double x0 = H(k + 1, k);
        const double alpha = x0 >= 0.0 ? -nrm : nrm;
        for (int i = 0; i < n; i++) v[i] = 0.0;
        v[k + 1] = x0 - alpha;
        for (int i = k + 2; i < n; i++) v[i] = H(i, k);
        double vv = 0.0;
        for (int i = k + 1; i < n; i++) vv += v[i] * v[i];
        if (vv == 0.0) continue;
        // H = P H P, Q = Q P with P = I - 2 v v^T / vv
        for (int j = 0; j < n; j++) {
            double s = 0.0;
            for (int i = k + 1; i < n; i++) s += v[i] * H(i, j);
            s *= 2.0 / vv;
            for (int i = k + 1; i < n; i++) H(i, j) -= s * v[i];
        }
        for (int i = 0; i < n; i++) {
            double s = 0.0;
            for (int j = k + 1; j < n; j++) s += H(i, j) * v[j];
            s *= 2.0 / vv;
            for (int j = k + 1; j < n; j++) H(i, j) -= s * v[j];
        }
        for (int i = 0; i < n; i++) {
            double s = 0.0;
            for (int j = k + 1; j < n; j++) s += Q(i, j) * v[j];
            s *= 2.0 / vv;
            for (int j = k + 1; j < n; j++) Q(i, j) -= s * v[j];
        }
        for (int i = k + 2; i < n; i++) H(i, k) = 0.0;
    }
}

}  // namespace

bool real_schur(int n, const double* A, double* Qout, double* Tout, double* resid) {
    const double eps = 2.220446049250313e-16;
    double amax = 0.0;
    for (int i = 0; i < n * n; i++) amax = std::fmax(amax, std::fabs(A[i]));
    if (!std::isfinite(amax)) return false;
    Mat H{n, std::vector<double>(A, A + (size_t)n * n)};
    Mat Q{n, std::vector<double>((size_t)n * n, 0.0)};
    for (int i = 0; i < n; i++) Q(i, i) = 1.0;
    if (amax > 0.0) hessenberg(H, Q);
    std::vector<double> cs(n), sn(n);
    int hi = n - 1, iter = 0, since = 0;
    while (hi > 0 && amax > 0.0) {
        int l = hi;
        while (l > 0 && std::fabs(H(l, l - 1)) > eps * (std::fabs(H(l - 1, l - 1)) + std::fabs(H(l, l)))) l--;
        if (l > 0) H(l, l - 1) = 0.0;
        if (l == hi) { hi--; since = 0; continue; }
        const double a = H(hi - 1, hi - 1), b = H(hi - 1, hi), c = H(hi, hi - 1), d = H(hi, hi);
        const double half = 0.5 * (a - d), disc = half * half + b * c;
        // a trailing 2 x 2 window with a complex pair (beyond rounding of a double real
        // eigenvalue) has no real Schur form
        if (l == hi - 1 && disc < -64.0 * eps * (half * half + std::fabs(b * c) + 0.25 * (a + d) * (a + d)))
            return false;
        // a defective (Jordan-like) double eigenvalue: the 2 x 2 window's subdiagonal stalls
        // near the unit roundoff instead of deflating; after 40 sweeps it is set to zero when
        // below 1e-8 of the diagonal (a perturbation of that size of the operator, which the
        // residual check below bounds)
        if (l == hi - 1 && since >= 40 && std::fabs(c) <= 1e-8 * (std::fabs(a) + std::fabs(d))) {
            H(hi, hi - 1) = 0.0;
            hi -= 2;
            since = 0;
            continue;
        }
        if (++iter > 100 * n) return false;
        // Wilkinson shift: the trailing block's eigenvalue closer to d (their mean for a pair
        // of equal or nearly complex eigenvalues); an exceptional shift every tenth sweep
        // without deflation
        double mu = 0.5 * (a + d);
        if (disc > 0.0) {
            const double sq = std::sqrt(disc);
            const double e1 = 0.5 * (a + d) + sq, e2 = 0.5 * (a + d) - sq;
            mu = std::fabs(e1 - d) < std::fabs(e2 - d) ? e1 : e2;
        }
        if (++since % 10 == 0 && hi >= 2) mu = d + std::fabs(H(hi, hi - 1)) + std::fabs(H(hi - 1, hi - 2));
        // shifted QR step on the active window l..hi as a similarity of the whole matrix:
        // the rotations are chosen from H - mu I restricted to the window and applied to all
        // of H (the shift cancels in Q^T H Q) and to Q
        double x = H(l, l) - mu, y = H(l + 1, l);
        for (int k = l; k < hi; k++) {
            const double r = std::hypot(x, y);
            const double cc = r == 0.0 ? 1.0 : x / r, ss = r == 0.0 ? 0.0 : y / r;
            rotate(H, Q, k, cc, ss, k == l ? l : k - 1, std::min(k + 2, hi));
            if (k + 1 < hi) {
                x = H(k + 1, k);
                y = H(k + 2, k);
            }
        }
    }
    // T = Q^T A Q from the iteration (lower part zero) and the residual of Q T Q^T - A
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            Tout[(size_t)i * n + j] = j >= i ? H(i, j) : 0.0;
            Qout[(size_t)i * n + j] = Q(i, j);
        }
    double off = 0.0;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            double s = 0.0;
            for (int k = 0; k < n; k++) {
                double qt = 0.0;
                for (int m = k; m < n; m++) qt += Tout[(size_t)k * n + m] * Q(j, m);
                s += Q(i, k) * qt;
            }
            off = std::fmax(off, std::fabs(s - A[(size_t)i * n + j]));
        }
    const double res = amax > 0.0 ? off / amax : off;
    if (resid) *resid = res;
    return res <= 1e-11;
}

}  // namespace gk
