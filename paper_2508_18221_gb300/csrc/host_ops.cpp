// Host-side construction of the grid operators and of the Kerr-Schild initial data.
//
// Differentiation matrices use barycentric Lagrange weights (Berrut & Trefethen 2004):
// D_ij = (w_j / w_i) / (x_i - x_j), D_ii = -sum_{j != i} D_ij, which is the same linear
// map as the paper's Chebyshev coefficient route (interpolate, chebder, evaluate).
// The Fourier first derivative on N (even) uniform nodes is the circulant matrix with
// row c_m = (-1)^m cot(m pi / N) / 2, c_0 = 0 (the (ik) multiplier with the Nyquist
// mode removed).  Modal filters are V diag(sigma) V^{-1} with the discrete Chebyshev
// transforms of the Lobatto and Gauss node sets, and a circulant row for phi.
#include "host_ops.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace gk {

static const double PI = 3.14159265358979323846;

std::vector<double> cgl_nodes(int n) {
    std::vector<double> x(n);
    for (int i = 0; i < n; i++) x[i] = -std::cos(i * PI / (n - 1));
    if (n % 2 == 1) x[n / 2] = 0.0;
    return x;
}

std::vector<double> gauss_nodes(int n) {
    std::vector<double> x(n);
    for (int k = 0; k < n; k++) x[k] = -std::cos((2 * k + 1) * PI / (2.0 * n));
    if (n % 2 == 1) x[n / 2] = 0.0;
    return x;
}

static std::vector<double> bary_matrix(const std::vector<double>& x, const std::vector<double>& w) {
    int n = (int)x.size();
    std::vector<double> D((size_t)n * n, 0.0);
    for (int i = 0; i < n; i++) {
        double s = 0.0;
        for (int j = 0; j < n; j++) {
            if (j == i) continue;
            double v = (w[j] / w[i]) / (x[i] - x[j]);
            D[(size_t)i * n + j] = v;
            s += v;
        }
        D[(size_t)i * n + i] = -s;
    }
    return D;
}

std::vector<double> cheb_lobatto_D(int n) {
    std::vector<double> x = cgl_nodes(n), w(n);
    for (int j = 0; j < n; j++) w[j] = ((j % 2) ? -1.0 : 1.0) * ((j == 0 || j == n - 1) ? 0.5 : 1.0);
    return bary_matrix(x, w);
}

std::vector<double> cheb_gauss_D(int n) {
    std::vector<double> x = gauss_nodes(n), w(n);
    for (int j = 0; j < n; j++) w[j] = ((j % 2) ? -1.0 : 1.0) * std::sin((2 * j + 1) * PI / (2.0 * n));
    return bary_matrix(x, w);
}

std::vector<double> fourier_D_row(int n) {
    std::vector<double> c(n, 0.0);
    for (int m = 1; m < n; m++) c[m] = 0.5 * ((m % 2) ? -1.0 : 1.0) / std::tan(m * PI / n);
    return c;
}

static double sigma(double k, double kmax, double alpha, double p) {
    return std::exp(-alpha * std::pow(std::fabs(k) / kmax, p));
}

// T_k(x_j) on the ascending Lobatto / Gauss nodes via the angle: x = -cos(t) = cos(pi - t)
static double Tk_lobatto(int k, int j, int n) { return std::cos(k * (PI - j * PI / (n - 1))); }
static double Tk_gauss(int k, int j, int n) { return std::cos(k * (PI - (2 * j + 1) * PI / (2.0 * n))); }

// inverse discrete Chebyshev transform coefficients: c_k = sum_j Vinv[k][j] u_j
static double vinv_lobatto(int k, int j, int n) {
    double ck = (k == 0 || k == n - 1) ? 2.0 : 1.0;
    double cj = (j == 0 || j == n - 1) ? 2.0 : 1.0;
    return 2.0 / ((n - 1) * ck * cj) * Tk_lobatto(k, j, n);
}
static double vinv_gauss(int k, int j, int n) {
    return (k == 0 ? 1.0 : 2.0) / n * Tk_gauss(k, j, n);
}

std::vector<double> cheb_filter_matrix(int n, bool lobatto, double alpha, double p) {
    std::vector<double> F((size_t)n * n, 0.0);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            double s = 0.0;
            for (int k = 0; k < n; k++) {
                double sg = sigma(k, n - 1, alpha, p);
                s += (lobatto ? Tk_lobatto(k, i, n) : Tk_gauss(k, i, n)) * sg *
                     (lobatto ? vinv_lobatto(k, j, n) : vinv_gauss(k, j, n));
            }
            F[(size_t)i * n + j] = s;
        }
    return F;
}

std::vector<double> fourier_filter_row(int n, double alpha, double p, bool dealias) {
    std::vector<double> f(n, 0.0);
    for (int m = 0; m < n; m++) {
        double s = 0.0;
        for (int k = 0; k < n; k++) {
            int kk = k <= n / 2 ? k : k - n;
            double sg = sigma(kk, n / 2.0, alpha, p);
            if (dealias && std::fabs((double)kk) > n / 3.0) sg = 0.0;
            s += sg * std::cos(2.0 * PI * kk * m / n);
        }
        f[m] = s / n;
    }
    return f;
}

// integrals of T_k over [-1, 1]
static double Tint(int k) { return (k % 2) ? 0.0 : 2.0 / (1.0 - (double)k * k); }

std::vector<double> quad_weights(int n, bool lobatto) {
    std::vector<double> w(n, 0.0);
    for (int j = 0; j < n; j++) {
        double s = 0.0;
        for (int k = 0; k < n; k++) s += Tint(k) * (lobatto ? vinv_lobatto(k, j, n) : vinv_gauss(k, j, n));
        w[j] = s;
    }
    return w;
}

// ---------------------------------------------------------------- Fourier theta
// Double-Fourier extension (the paper's Fourier theta derivative on theta_k = (k + 1/2) pi
// / n): the 2n extended nodes hold u_k (k < n) and s u'_{2n-1-k} (n <= k < 2n), u' the
// line at phi + pi and s the component's parity, so with the circulant operator
// C_ij = c[(i - j) mod 2n] of the extended nodes
//   (C g)_i = sum_k A_ik u_k + s sum_k B_ik u'_k,  A_ik = c[(i - k) mod 2n],
//   B_ik = c[(i + k + 1) mod 2n].
// Writing u = p + m, u' = p - m (p, m the half sum and half difference of the phi pair)
// gives (C g)_i = ((A + s B) p)_i + ((A - s B) m)_i at phi and the same with -m at
// phi + pi: the sums take A + B for s = +1 (A - B for s = -1), the differences the other.
// scale multiplies both (exact for a power of two): 1/2 when the fold forms the plain sum
// and difference of the pair, 1 on a line of definite parity.
void theta_extension_ops(const std::vector<double>& c, int n, std::vector<double>* even,
                         std::vector<double>* odd, double scale) {
    const int n2 = 2 * n;
    even->assign((size_t)n * n, 0.0);
    odd->assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; i++)
        for (int k = 0; k < n; k++) {
            const double a = c[((i - k) % n2 + n2) % n2];
            const double b = c[(i + k + 1) % n2];
            (*even)[(size_t)i * n + k] = scale * (a + b);
            (*odd)[(size_t)i * n + k] = scale * (a - b);
        }
}

// ---------------------------------------------------------------- reflection split
// Index pairs and fixed points of the node reflection (see kernels_eo.cu):
// kind 0 (Chebyshev nodes): pairs (ip, N-1-ip), ip < N/2; fixed N/2 when N is odd.
// kind 1 (Fourier nodes):   pairs (ip+1, N-1-ip), ip < N/2-1; fixed 0 and N/2.
static void split_sets(int N, int kind, std::vector<int>& lo, std::vector<int>& hi, std::vector<int>& fx) {
    lo.clear(); hi.clear(); fx.clear();
    int np = kind == 0 ? N / 2 : N / 2 - 1;
    for (int ip = 0; ip < np; ip++) {
        lo.push_back(kind == 0 ? ip : ip + 1);
        hi.push_back(N - 1 - ip);
    }
    if (kind == 0) { if (N % 2) fx.push_back(N / 2); }
    else { fx.push_back(0); fx.push_back(N / 2); }
}

std::vector<double> split_operator(const std::vector<double>& M, int N, int kind) {
    std::vector<int> lo, hi, fx;
    split_sets(N, kind, lo, hi, fx);
    int np = (int)lo.size(), nf = (int)fx.size();
    std::vector<double> out;
    out.reserve((size_t)2 * np * np + 2 * np * nf + nf * nf);
    auto m = [&](int i, int j) { return M[(size_t)i * N + j]; };
    for (int i = 0; i < np; i++)      // E
        for (int j = 0; j < np; j++) out.push_back(0.5 * (m(lo[i], lo[j]) + m(lo[i], hi[j])));
    for (int i = 0; i < np; i++)      // O
        for (int j = 0; j < np; j++) out.push_back(0.5 * (m(lo[i], lo[j]) - m(lo[i], hi[j])));
    for (int i = 0; i < np; i++)      // C: fixed-point columns of the pair rows
        for (int f = 0; f < nf; f++) out.push_back(m(lo[i], fx[f]));
    for (int f = 0; f < nf; f++)      // F: fixed-point rows against the pair columns
        for (int j = 0; j < np; j++) out.push_back(m(fx[f], lo[j]));
    for (int f = 0; f < nf; f++)      // G: fixed-point block
        for (int g = 0; g < nf; g++) out.push_back(m(fx[f], fx[g]));
    return out;
}

// ---------------------------------------------------------------- tensor-core images
static uint16_t bf16_rne(double x) {
    float f = (float)x;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
static double bf16_val(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return (double)f;
}
static uint32_t tf32_rne(double x) {
    float f = (float)x;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0xFFFu + ((u >> 13) & 1u);
    return u & ~0x1FFFu;
}

std::vector<uint8_t> tc_operator_image(const std::vector<double>& D, int N, int tf32) {
    const int Kp = (N + 15) / 16 * 16, Np = Kp;
    const int es = tf32 ? 4 : 2, per = 16 / es, kcores = Kp * es / 16, nsl = tf32 ? 1 : 3;
    const size_t slice = (size_t)Np * Kp * es;
    std::vector<uint8_t> img(slice * nsl, 0);
    for (int n = 0; n < N; n++)
        for (int k = 0; k < N; k++) {
            size_t off = (size_t)((n >> 3) * kcores + k / per) * 128 + (n & 7) * 16 + (k % per) * es;
            double x = D[(size_t)n * N + k];
            if (tf32) {
                uint32_t u = tf32_rne(x);
                std::memcpy(&img[off], &u, 4);
            } else {
                uint16_t b1 = bf16_rne(x);
                double r1 = x - bf16_val(b1);
                uint16_t b2 = bf16_rne(r1);
                uint16_t b3 = bf16_rne(r1 - bf16_val(b2));
                std::memcpy(&img[off], &b1, 2);
                std::memcpy(&img[slice + off], &b2, 2);
                std::memcpy(&img[2 * slice + off], &b3, 2);
            }
        }
    return img;
}

// Digit slices of the operator rows for the FP64-accurate tensor-core contraction.  Row
// n of scale * D gets the exponent F_n (largest biased exponent of the row, 0 for a zero
// row); Y = round(x 2^(1076 - F_n)) is a signed integer with |Y| <= 2^54, and the bytes of
// Y + 0x80808080808080 minus 128 are its balanced base-256 digits c_1..c_7 (most
// significant first).  Slice l holds c_l 2^(-8 (l - 1)), exact in BF16.
// IEEE binary16 bits of an integer d in [-128, 127] (exact: at most 8 significant bits)
static uint16_t half_of_digit(int d) {
    if (d == 0) return 0;
    const uint16_t sgn = d < 0 ? 0x8000 : 0;
    const int a = d < 0 ? -d : d;
    int e = 0;
    while ((a >> (e + 1)) != 0) e++;                      // a in [2^e, 2^(e+1))
    return (uint16_t)(sgn | ((e + 15) << 10) | ((a - (1 << e)) << (10 - e)));
}

std::vector<uint8_t> fx_operator_image(const std::vector<double>& D, int N, double scale, int Np, int Kp,
                                       int KC) {
    const int nch = Kp / KC, kcores = KC / 8, Npp = Np > 64 ? 64 : Np;
    const size_t slice = (size_t)Np * KC * 2, chunk = 7 * slice;
    const size_t bytes = ((size_t)nch * chunk + (size_t)Np * 4 + 15) / 16 * 16;
    std::vector<uint8_t> img(bytes, 0);
    std::vector<int32_t> fexp(Np, 0);
    for (int n = 0; n < N; n++) {
        int F = 0;
        for (int k = 0; k < N; k++) {
            const double x = D[(size_t)n * N + k] * scale;
            if (x != 0.0) {
                int ex;
                std::frexp(x, &ex);
                F = std::max(F, ex + 1022);
            }
        }
        fexp[n] = F;
        if (F <= 0) continue;
        for (int k = 0; k < N; k++) {
            const double x = D[(size_t)n * N + k] * scale;
            const long long Y = std::llround(std::ldexp(x, 1076 - F));
            const unsigned long long Z = (unsigned long long)(Y + 0x80808080808080LL);
            const int kc = k / KC, kk = k % KC;
            for (int q = 1; q <= 7; q++) {
                const int digit = (int)((Z >> (8 * (7 - q))) & 0xFF) - 128;
                const uint16_t b = half_of_digit(digit);
                // row of the chunk's tall B matrix: pass p (Npp = min(Np, 64) output rows),
                // then slice, then the row within the pass
                const int row = ((n / Npp) * 7 + (q - 1)) * Npp + n % Npp;
                const size_t off = (size_t)kc * chunk + ((size_t)((row >> 3) * kcores + (kk >> 3))) * 128 +
                                   (row & 7) * 16 + (kk & 7) * 2;
                std::memcpy(&img[off], &b, 2);
            }
        }
    }
    std::memcpy(&img[(size_t)nch * chunk], fexp.data(), (size_t)Np * 4);
    return img;
}

std::vector<double> circulant(const std::vector<double>& row) {
    int n = (int)row.size();
    std::vector<double> M((size_t)n * n);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) M[(size_t)i * n + j] = row[((i - j) % n + n) % n];
    return M;
}

// ---------------------------------------------------------------- Kerr-Schild data
// forward-mode dual number for derivatives of the closed-form Kerr-Schild 3+1 fields
struct Dn {
    double v, d;
    Dn(double a = 0.0, double b = 0.0) : v(a), d(b) {}
};
static inline Dn operator+(Dn a, Dn b) { return Dn(a.v + b.v, a.d + b.d); }
static inline Dn operator-(Dn a, Dn b) { return Dn(a.v - b.v, a.d - b.d); }
static inline Dn operator-(Dn a) { return Dn(-a.v, -a.d); }
static inline Dn operator*(Dn a, Dn b) { return Dn(a.v * b.v, a.d * b.v + a.v * b.d); }
static inline Dn operator/(Dn a, Dn b) { return Dn(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
static inline Dn dsin(Dn a) { return Dn(std::sin(a.v), std::cos(a.v) * a.d); }
static inline Dn dcos(Dn a) { return Dn(std::cos(a.v), -std::sin(a.v) * a.d); }
static inline Dn dsqrtn(Dn a) { double s = std::sqrt(a.v); return Dn(s, 0.5 * a.d / s); }
static inline Dn dlog(Dn a) { return Dn(std::log(a.v), a.d / a.v); }
static inline Dn dexp(Dn a) { double e = std::exp(a.v); return Dn(e, e * a.d); }
static inline Dn dpow(Dn a, double q) { double v = std::pow(a.v, q); return Dn(v, q * v / a.v * a.d); }

// Closed forms derived from the line element (H = M r / Sigma):
// gamma_rr = 1+2H, gamma_rph = -a s^2 (1+2H), gamma_thth = Sigma,
// gamma_phph = s^2 (Sigma + a^2 s^2 (1+2H)), beta_i = (2H, 0, -2 a H s^2),
// beta^i = (2H/(1+2H), 0, 0), alpha = (1+2H)^{-1/2}.
static void ks_fields(double M, double a, Dn r, Dn th, Dn gam[3][3], Dn beta_d[3], Dn beta_u[3],
                      Dn* alpha) {
    Dn c = dcos(th), s = dsin(th);
    Dn s2 = s * s;
    Dn sig = r * r + Dn(a * a) * c * c;
    Dn H = Dn(M) * r / sig;
    Dn one2H = Dn(1.0) + Dn(2.0) * H;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) gam[i][j] = Dn(0.0);
    gam[0][0] = one2H;
    gam[0][2] = gam[2][0] = -(Dn(a) * s2 * one2H);
    gam[1][1] = sig;
    gam[2][2] = s2 * (sig + Dn(a * a) * s2 * one2H);
    beta_d[0] = Dn(2.0) * H;
    beta_d[1] = Dn(0.0);
    beta_d[2] = -(Dn(2.0 * a) * H * s2);
    beta_u[0] = Dn(2.0) * H / one2H;
    beta_u[1] = Dn(0.0);
    beta_u[2] = Dn(0.0);
    *alpha = Dn(1.0) / dsqrtn(one2H);
}

static double det3h(const double g[3][3]) {
    return g[0][0] * (g[1][1] * g[2][2] - g[1][2] * g[2][1]) -
           g[0][1] * (g[1][0] * g[2][2] - g[1][2] * g[2][0]) +
           g[0][2] * (g[1][0] * g[2][1] - g[1][1] * g[2][0]);
}
static void inv3h(const double g[3][3], double gi[3][3]) {
    double d = det3h(g);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            int r0 = (j + 1) % 3, r1 = (j + 2) % 3, c0 = (i + 1) % 3, c1 = (i + 2) % 3;
            gi[i][j] = (g[r0][c0] * g[r1][c1] - g[r0][c1] * g[r1][c0]) / d;
        }
}

// conformal metric gammatilde_ij(r, th) = gamma_ij / det(gamma)^{1/3} with dual derivative
static void ks_conformal(double M, double a, Dn r, Dn th, Dn gt[3][3]) {
    Dn gam[3][3], bd[3], bu[3], al;
    ks_fields(M, a, r, th, gam, bd, bu, &al);
    Dn det = gam[0][0] * (gam[1][1] * gam[2][2] - gam[1][2] * gam[2][1]) -
             gam[0][1] * (gam[1][0] * gam[2][2] - gam[1][2] * gam[2][0]) +
             gam[0][2] * (gam[1][0] * gam[2][1] - gam[1][1] * gam[2][0]);
    Dn f = dpow(det, -1.0 / 3.0);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) gt[i][j] = gam[i][j] * f;
}

void ks_bssn_point(double M, double a, double r, double th, double out[24]) {
    // values and (r, theta) derivatives of gamma_ij and beta_i
    double g[3][3], dg[3][3][3] = {}, bdv[3], dbd[3][3] = {}, alpha = 0.0;
    for (int dir = 0; dir < 2; dir++) {
        Dn R(r, dir == 0 ? 1.0 : 0.0), T(th, dir == 1 ? 1.0 : 0.0);
        Dn gam[3][3], bd[3], bu[3], al;
        ks_fields(M, a, R, T, gam, bd, bu, &al);
        for (int i = 0; i < 3; i++) {
            for (int j = 0; j < 3; j++) { g[i][j] = gam[i][j].v; dg[dir][i][j] = gam[i][j].d; }
            bdv[i] = bd[i].v;
            dbd[dir][i] = bd[i].d;
        }
        alpha = al.v;
    }
    double gi[3][3];
    inv3h(g, gi);
    // Christoffels Gamma^k_ij of gamma (phi derivatives vanish: axisymmetry)
    double Cl[3][3][3], Cu[3][3][3];
    for (int k = 0; k < 3; k++)
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) Cl[k][i][j] = 0.5 * (dg[i][k][j] + dg[j][k][i] - dg[k][i][j]);
    for (int k = 0; k < 3; k++)
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double s = 0.0;
                for (int l = 0; l < 3; l++) s += gi[k][l] * Cl[l][i][j];
                Cu[k][i][j] = s;
            }
    // K_ij = (d_i beta_j + d_j beta_i - 2 Gamma^k_ij beta_k) / (2 alpha)
    double Kij[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double cb = 0.0;
            for (int k = 0; k < 3; k++) cb += Cu[k][i][j] * bdv[k];
            Kij[i][j] = (dbd[i][j] + dbd[j][i] - 2.0 * cb) / (2.0 * alpha);
        }
    double det = det3h(g);
    double phi = std::log(det) / 12.0;
    double e4m = std::exp(-4.0 * phi);
    double K = 0.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) K += gi[i][j] * Kij[i][j];
    // conformal metric derivatives and Gammatilde^i = gt^jk Gammatilde^i_jk
    double gt[3][3], dgt[3][3][3] = {};
    for (int dir = 0; dir < 2; dir++) {
        Dn R(r, dir == 0 ? 1.0 : 0.0), T(th, dir == 1 ? 1.0 : 0.0);
        Dn c[3][3];
        ks_conformal(M, a, R, T, c);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) { gt[i][j] = c[i][j].v; dgt[dir][i][j] = c[i][j].d; }
    }
    double gti[3][3];
    inv3h(gt, gti);
    double Gam[3];
    for (int i = 0; i < 3; i++) {
        double s = 0.0;
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++) {
                double ct = 0.0;
                for (int l = 0; l < 3; l++)
                    ct += gti[i][l] * 0.5 * (dgt[j][l][k] + dgt[k][l][j] - dgt[l][j][k]);
                s += gti[j][k] * ct;
            }
        Gam[i] = s;
    }
    const int sp[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    for (int n = 0; n < 6; n++) {
        int i = sp[n][0], j = sp[n][1];
        out[0 + n] = e4m * g[i][j];
        out[7 + n] = e4m * (Kij[i][j] - g[i][j] * K / 3.0);
    }
    out[6] = phi;
    out[13] = K;
    for (int i = 0; i < 3; i++) out[14 + i] = Gam[i];
    out[17] = alpha;
    out[18] = 2.0 * (M * r / (r * r + a * a * std::cos(th) * std::cos(th)));
    out[18] = out[18] / (1.0 + out[18]);
    out[19] = 0.0;
    out[20] = 0.0;
    out[21] = out[22] = out[23] = 0.0;
}

// Conserved (undensitized) variables from primitives in the Eulerian form:
// Z = rho h W^2, S_j = (Z + B^2) v_j - (v.B) B_j, tau = Z + B^2 - p - (B^2/W^2 + (v.B)^2)/2 - D
void prim_to_cons_point(double rho, double p, const double v_u[3], const double B_u[3],
                        const double g[3][3], double gam_eos, double* D, double S_d[3],
                        double* tau) {
    double v_d[3], B_d[3];
    for (int i = 0; i < 3; i++) {
        v_d[i] = g[i][0] * v_u[0] + g[i][1] * v_u[1] + g[i][2] * v_u[2];
        B_d[i] = g[i][0] * B_u[0] + g[i][1] * B_u[1] + g[i][2] * B_u[2];
    }
    double v2 = v_d[0] * v_u[0] + v_d[1] * v_u[1] + v_d[2] * v_u[2];
    double W = 1.0 / std::sqrt(1.0 - v2);
    double eps = p / ((gam_eos - 1.0) * rho);
    double h = 1.0 + eps + p / rho;
    double Z = rho * h * W * W;
    double B2 = B_d[0] * B_u[0] + B_d[1] * B_u[1] + B_d[2] * B_u[2];
    double vB = v_d[0] * B_u[0] + v_d[1] * B_u[1] + v_d[2] * B_u[2];
    *D = rho * W;
    for (int j = 0; j < 3; j++) S_d[j] = (Z + B2) * v_d[j] - vB * B_d[j];
    *tau = Z + B2 - p - 0.5 * (B2 / (W * W) + vB * vB) - rho * W;
}

void metric_from_bssn_point(const double* bssn, double g[3][3], double* sqg) {
    double e4 = std::exp(4.0 * bssn[6]);
    const int sidx[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) g[i][j] = e4 * bssn[sidx[i][j]];
    *sqg = std::sqrt(det3h(g));
}

}  // namespace gk
