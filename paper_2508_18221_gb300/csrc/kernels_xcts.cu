// Approximate XCTS initial data (paper: "Initial Data: Approximate XCTS Solution"): the
// conformal Hamiltonian constraint  lap psi = -2 pi rho psi^5  with the flat conformal
// metric, solved by the paper's fixed-point relaxation psi_{k+1} = L^-1(-2 pi rho psi_k^5).
//
// Discretisation (the same readings as the evolution grid): element-local Chebyshev
// derivatives in r, the double-Fourier theta derivatives of the Fourier theta basis, the
// Fourier series in phi.  The Laplacian separates in phi: for the real modes
// cos(m phi), sin(m phi) (m = 0..N_phi/2) it is, on the (r, theta) nodes of all elements,
//   L_m = d_rr + (2/r) d_r + (D2_s + cot(theta) D1_s - m'^2 / sin^2 theta) / r^2,
// with D1_s, D2_s the theta derivatives for the mode's extension parity s = (-1)^m (a scalar
// has parity +1, and its phi + pi partner carries (-1)^m) and m'^2 = m^2 except at the
// Nyquist mode, whose phi derivative the grid zeroes.  The rows of the element end nodes
// carry the boundary and interface conditions: inner node of element 0 d_r psi =
// -M / (2 r_min^2) (the puncture's derivative), outer node of the last element
// psi + r_max d_r psi = 1 (Robin, psi - 1 ~ 1/r), at a shared interface the left copy
// psi_L = psi_R and the right copy d_r psi_L = d_r psi_R.
//
// The operator of one mode is a Kronecker sum: L_m = R (x) I + diag(S) (x) Theta_m, with R the
// radial operator over all elements (the end rows carrying the conditions, which act on
// each theta node alone), S = 1/r^2 on the rows of interior nodes and 0 on end rows, and
// Theta_m the N_theta x N_theta angular operator above.  With the real Schur form
// Theta_m = Q T Q^T (Q orthogonal, T upper triangular; host_eig.cpp), L_m = (I (x) Q)
// (R (x) I + diag(S) (x) T)(I (x) Q^T), and the middle factor is block upper triangular in the
// Schur index j: the solve is a back substitution over j, each step one radial system
// R + T_jj diag(S) of E N_r unknowns -- the same solution as the dense (E N_r N_theta)^2
// system per mode, for O(N_theta (E N_r)^3) work instead of O((E N_r N_theta)^3), and with an
// orthogonal change of basis whatever the angular operator's eigenvectors (at some theta
// orders two of them nearly coincide).  GPU work: one kernel forms and inverts every radial
// system (Gauss-Jordan with partial pivoting, one CTA per system, once); per iteration one
// kernel forms the source and the forward real Fourier transform in phi, one applies Q^T to
// every theta line, one runs the back substitution (a CTA per mode and cos / sin column:
// y_j = inverse times G_j, then T_ij S y_j subtracted from the steps i < j),
// one applies Q, and one takes the inverse transform with the change
// max |psi_{k+1} - psi_k| (block maxima, one atomic per block).
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "grmhd_internal.h"
#include "host_ops.h"

namespace gk {

namespace {

struct XDev {
    int E, Nr, Nt, Np, n, nmodes, nr;   // n = E Nr Nt nodes per phi line set, nr = E Nr
    const double* cs;     // [nmodes][Np] cos(2 pi m l / Np)
    const double* sn;     // [nmodes][Np] sin(2 pi m l / Np)
    const double* bval;   // [nr] boundary data of the end rows (phi mode 0, cosine)
    const int* end;       // [nr] 1 for an end (boundary / interface) row
};

// right-hand sides of all modes, column-major n x 2 per mode (cos, sin):
// a_m = c_m / Np sum_l F_l cos(m phi_l), b_m = 2 / Np sum_l F_l sin(m phi_l),
// c_0 = c_{Np/2} = 1, else 2; F = -2 pi rho psi^5 on PDE rows, boundary rows transformed
// exactly (their data are constant in phi)
__global__ void k_xcts_forward(XDev x, const double* __restrict__ rho, const double* __restrict__ psi,
                               double* __restrict__ B) {
    const long long total = (long long)x.n * x.nmodes;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(t / x.n), q = (int)(t - (long long)m * x.n);
        const int ri = q / x.Nt;              // radial node over all elements
        double a = 0.0, b = 0.0;
        if (x.end[ri]) {
            a = m == 0 ? x.bval[ri] : 0.0;
        } else {
            const double* rq = rho + (size_t)q * x.Np;
            const double* pq = psi + (size_t)q * x.Np;
            const double* cm = x.cs + (size_t)m * x.Np;
            const double* sm = x.sn + (size_t)m * x.Np;
            for (int l = 0; l < x.Np; l++) {
                const double p2 = pq[l] * pq[l];
                const double f = -2.0 * M_PI * rq[l] * (p2 * p2 * pq[l]);
                a = fma(f, cm[l], a);
                b = fma(f, sm[l], b);
            }
            const double c = (m == 0 || 2 * m == x.Np) ? 1.0 : 2.0;
            a *= c / x.Np;
            b *= 2.0 / x.Np;
        }
        B[(size_t)m * 2 * x.n + q] = a;
        B[(size_t)m * 2 * x.n + x.n + q] = b;
    }
}

// psi = sum_m a_m cos(m phi) + b_m sin(m phi); max |change| into *chg (bit pattern of a
// non-negative double: the integer order is the value order)
__global__ void k_xcts_inverse(XDev x, const double* __restrict__ B, double* __restrict__ psi,
                               unsigned long long* chg) {
    __shared__ double red[8];
    const long long total = (long long)x.n * x.Np;
    double mx = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(t / x.Np), l = (int)(t - (long long)q * x.Np);
        double v = 0.0;
        for (int m = 0; m < x.nmodes; m++) {
            const double* Bm = B + (size_t)m * 2 * x.n;
            v = fma(Bm[q], x.cs[(size_t)m * x.Np + l], v);
            v = fma(Bm[x.n + q], x.sn[(size_t)m * x.Np + l], v);
        }
        const double dv = fabs(v - psi[t]);
        mx = dv == dv ? fmax(mx, dv) : __longlong_as_double(0x7ff0000000000000LL);  // NaN counts as +inf
        psi[t] = v;
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) mx = fmax(mx, red[w]);
        atomicMax(chg, (unsigned long long)__double_as_longlong(mx));
    }
}

// Form R + lam diag(S) of one radial system (one CTA per system: sys = m N_theta + j) next to
// the identity, [A | I] (row-major nr x 2 nr), and reduce it by Gauss-Jordan elimination with
// partial pivoting to [I | A^-1]; info[sys] = 1 for an exactly zero pivot.  The inverse turns
// every radial solve of the fixed-point iteration into one matrix-vector product.
__global__ void __launch_bounds__(256) k_xcts_radial_inverse(XDev x, const double* __restrict__ R,
                                                             const double* __restrict__ S,
                                                             const double* __restrict__ lam,
                                                             double* __restrict__ W_all, int* __restrict__ info) {
    __shared__ double s_val[8];
    __shared__ int s_idx[8];
    __shared__ int s_p;
    const int sys = blockIdx.x, nr = x.nr, w2 = 2 * nr, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    double* W = W_all + (size_t)sys * nr * w2;
    const double lj = lam[sys];
    for (int idx = tid; idx < nr * w2; idx += blockDim.x) {
        const int i = idx / w2, j = idx - i * w2;
        W[idx] = j < nr ? R[(size_t)i * nr + j] + (i == j ? lj * S[i] : 0.0) : (j - nr == i ? 1.0 : 0.0);
    }
    __syncthreads();
    for (int k = 0; k < nr; k++) {
        // pivot: the largest |W[i][k]|, i >= k (the smallest index among equals)
        double best = -1.0;
        int bi = k;
        for (int i = k + tid; i < nr; i += blockDim.x) {
            const double a = fabs(W[(size_t)i * w2 + k]);
            if (a > best) { best = a; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) { s_val[w] = best; s_idx[w] = bi; }
        __syncthreads();
        if (tid == 0) {
            double b = s_val[0];
            int p = s_idx[0];
            for (int q = 1; q < (int)(blockDim.x >> 5); q++)
                if (s_val[q] > b || (s_val[q] == b && s_idx[q] < p)) { b = s_val[q]; p = s_idx[q]; }
            s_p = p;
            if (!(b > 0.0)) info[sys] = 1;
        }
        __syncthreads();
        const int p = s_p;
        // swap rows k and p, then scale row k by 1 / pivot (columns k.. : the left part before
        // k is already the identity)
        if (p != k)
            for (int j = k + tid; j < w2; j += blockDim.x) {
                const double t = W[(size_t)k * w2 + j];
                W[(size_t)k * w2 + j] = W[(size_t)p * w2 + j];
                W[(size_t)p * w2 + j] = t;
            }
        __syncthreads();
        const double pv = W[(size_t)k * w2 + k];
        __syncthreads();
        if (pv != 0.0)
            for (int j = k + tid; j < w2; j += blockDim.x) W[(size_t)k * w2 + j] /= pv;
        __syncthreads();
        // eliminate column k from every other row (columns k + 1 ..)
        const int cols = w2 - k - 1;
        for (int t = tid; t < (nr - 1) * cols; t += blockDim.x) {
            int i = t / cols;
            const int j = k + 1 + (t - i * cols);
            i += i >= k;                                   // every row but k
            W[(size_t)i * w2 + j] -= W[(size_t)i * w2 + k] * W[(size_t)k * w2 + j];
        }
        __syncthreads();
        for (int i = tid; i < nr; i += blockDim.x)
            if (i != k) W[(size_t)i * w2 + k] = 0.0;
        __syncthreads();
    }
}

// theta transforms of every (mode, cos / sin) block with the mode's orthogonal Q (row-major,
// Q[k][j]): forward G[m][c][j][r] = sum_k Q_m[k][j] B[m][c][r Nt + k] (Q^T); backward
// B[m][c][r Nt + k] = sum_j Q_m[k][j] G[m][c][j][r] (Q)
__global__ void k_xcts_theta(XDev x, const double* __restrict__ Q, const double* __restrict__ in,
                             double* __restrict__ out, int forward) {
    const int Nt = x.Nt, nr = x.nr;
    const long long total = (long long)x.nmodes * 2 * Nt * nr;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int mc = (int)(t / ((long long)Nt * nr));
        const int rem = (int)(t - (long long)mc * Nt * nr);
        const int m = mc >> 1;
        const double* Qm = Q + (size_t)m * Nt * Nt;
        if (forward) {
            const int j = rem / nr, r = rem - j * nr;                   // out: G[mc][j][r]
            const double* b = in + (size_t)mc * x.n + (size_t)r * Nt;
            double v = 0.0;
            for (int k = 0; k < Nt; k++) v = fma(Qm[k * Nt + j], b[k], v);
            out[t] = v;
        } else {
            const int r = rem / Nt, k = rem - r * Nt;                   // out: B[mc][r Nt + k]
            const double* gmc = in + (size_t)mc * Nt * nr;
            double v = 0.0;
            for (int j = 0; j < Nt; j++) v = fma(Qm[k * Nt + j], gmc[(size_t)j * nr + r], v);
            out[(size_t)mc * x.n + rem] = v;
        }
    }
}

// Back substitution over the Schur index for one (mode, cos / sin) column (one CTA): for
// j = N_theta - 1 .. 0, y_j = (R + T_jj S)^-1 G_j with the inverse from
// k_xcts_radial_inverse (a thread per radial row), then G_i -= T_ij S y_j for every i < j.
// y overwrites G.
__global__ void __launch_bounds__(256) k_xcts_schur_solve(XDev x, const double* __restrict__ W_all,
                                                          const double* __restrict__ T,
                                                          const double* __restrict__ S, double* __restrict__ G) {
    extern __shared__ double g_s[];                  // [nr] right-hand side, then [nr] y
    const int nr = x.nr, Nt = x.Nt, tid = threadIdx.x, w2 = 2 * nr;
    const int mc = blockIdx.x, m = mc >> 1;
    const double* Tm = T + (size_t)m * Nt * Nt;
    double* Gm = G + (size_t)mc * Nt * nr;
    double* y = g_s + nr;
    for (int j = Nt - 1; j >= 0; j--) {
        double* g = Gm + (size_t)j * nr;
        for (int r = tid; r < nr; r += blockDim.x) g_s[r] = g[r];
        __syncthreads();
        const double* Ainv = W_all + (size_t)(m * Nt + j) * nr * w2 + nr;   // right half of [I | A^-1]
        for (int r = tid; r < nr; r += blockDim.x) {
            const double* row = Ainv + (size_t)r * w2;
            double v = 0.0;
            for (int k = 0; k < nr; k++) v = fma(row[k], g_s[k], v);
            y[r] = v;
            g[r] = v;
        }
        __syncthreads();
        for (int t = tid; t < j * nr; t += blockDim.x) {
            const int i = t / nr, r = t - i * nr;
            Gm[(size_t)i * nr + r] -= Tm[i * Nt + j] * S[r] * y[r];
        }
        __syncthreads();
    }
}

template <class T>
cudaError_t xalloc(T** p, size_t n) { return cudaMalloc((void**)p, n * sizeof(T) + 16); }

}  // namespace

int xcts_solve(const XctsOps& o, const double* rho_host, double* psi_host, int iters, double tol,
               double* changes, double* stats, cudaStream_t s, char* msg, size_t msglen) {
    const auto t_setup0 = std::chrono::steady_clock::now();
    const int nr = o.E * o.Nr, Nt = o.Nt, n = nr * Nt, nmodes = o.Np / 2 + 1, nsys = nmodes * Nt;
    const long long P = (long long)n * o.Np;
    // ---- host: radial operator R, S and the angular eigendecompositions
    std::vector<double> R((size_t)nr * nr, 0.0), S(nr, 0.0), bval(nr, 0.0);
    std::vector<int> endr(nr, 0);
    for (int e = 0; e < o.E; e++) {
        const double* Dre = o.Dr.data() + (size_t)e * o.Nr * o.Nr;
        const double* Drre = o.Drr.data() + (size_t)e * o.Nr * o.Nr;
        for (int i = 0; i < o.Nr; i++) {
            const int row = e * o.Nr + i;
            double* Rrow = R.data() + (size_t)row * nr;
            if (i == 0) {
                endr[row] = 1;
                for (int i2 = 0; i2 < o.Nr; i2++) Rrow[e * o.Nr + i2] += Dre[i2];
                if (e > 0)
                    for (int i2 = 0; i2 < o.Nr; i2++)
                        Rrow[(e - 1) * o.Nr + i2] -= o.Dr[((size_t)(e - 1) * o.Nr + o.Nr - 1) * o.Nr + i2];
                else
                    bval[row] = -o.M / (2.0 * o.r_min * o.r_min);
            } else if (i == o.Nr - 1) {
                endr[row] = 1;
                if (e == o.E - 1) {
                    for (int i2 = 0; i2 < o.Nr; i2++) Rrow[e * o.Nr + i2] += o.r_max * Dre[(size_t)(o.Nr - 1) * o.Nr + i2];
                    Rrow[row] += 1.0;
                    bval[row] = 1.0;
                } else {
                    Rrow[row] += 1.0;
                    Rrow[(e + 1) * o.Nr] -= 1.0;
                }
            } else {
                const double r = o.r[row];
                for (int i2 = 0; i2 < o.Nr; i2++)
                    Rrow[e * o.Nr + i2] = Drre[(size_t)i * o.Nr + i2] + 2.0 / r * Dre[(size_t)i * o.Nr + i2];
                S[row] = 1.0 / (r * r);
            }
        }
    }
    std::vector<double> lam((size_t)nsys), Qs((size_t)nmodes * Nt * Nt), Ts((size_t)nmodes * Nt * Nt);
    std::vector<double> Th((size_t)Nt * Nt);
    for (int m = 0; m < nmodes; m++) {
        const int sidx = m & 1;
        const double mm = (2 * m == o.Np) ? 0.0 : (double)m * m;
        for (int k = 0; k < Nt; k++) {
            const double st = std::sin(o.th[k]), ct = std::cos(o.th[k]);
            for (int k2 = 0; k2 < Nt; k2++) {
                double a = o.D2[((size_t)sidx * Nt + k) * Nt + k2] + ct / st * o.D1[((size_t)sidx * Nt + k) * Nt + k2];
                if (k2 == k) a -= mm / (st * st);
                Th[(size_t)k * Nt + k2] = a;
            }
        }
        double res = 0.0;
        double* Tm = Ts.data() + (size_t)m * Nt * Nt;
        if (!real_schur(Nt, Th.data(), Qs.data() + (size_t)m * Nt * Nt, Tm, &res)) {
            snprintf(msg, msglen, "XCTS solve: the angular operator of phi mode %d has no real Schur form "
                                  "(residual %.2e)", m, res);
            return GRMHD_EUNSUPPORTED;
        }
        for (int j = 0; j < Nt; j++) lam[(size_t)m * Nt + j] = Tm[(size_t)j * Nt + j];
    }
    std::vector<double> cs((size_t)nmodes * o.Np), sn((size_t)nmodes * o.Np);
    for (int m = 0; m < nmodes; m++)
        for (int l = 0; l < o.Np; l++) {
            const double a = 2.0 * M_PI * ((long long)m * l % o.Np) / o.Np;
            cs[(size_t)m * o.Np + l] = std::cos(a);
            sn[(size_t)m * o.Np + l] = std::sin(a);
        }
    double *dR = nullptr, *dS = nullptr, *dlam = nullptr, *dQ = nullptr, *dT = nullptr, *dbv = nullptr,
           *dcs = nullptr, *dsn = nullptr, *dA = nullptr, *dB = nullptr, *dG = nullptr, *drho = nullptr,
           *dpsi = nullptr;
    int *dinfo = nullptr, *dend = nullptr;
    unsigned long long* dchg = nullptr;
    int st = GRMHD_OK;
    cudaEvent_t e1 = nullptr, e2 = nullptr;
    auto fail = [&](int code, const char* what) {
        if (st == GRMHD_OK) {
            st = code;
            snprintf(msg, msglen, "XCTS solve: %s", what);
        }
        return code;
    };
    do {
        if (xalloc(&dR, R.size()) || xalloc(&dS, S.size()) || xalloc(&dlam, lam.size()) || xalloc(&dQ, Qs.size()) ||
            xalloc(&dT, Ts.size()) || xalloc(&dbv, bval.size()) || xalloc(&dend, endr.size()) ||
            xalloc(&dcs, cs.size()) || xalloc(&dsn, sn.size()) || xalloc(&dA, (size_t)nsys * nr * 2 * nr) ||
            xalloc(&dB, (size_t)2 * n * nmodes) || xalloc(&dG, (size_t)2 * n * nmodes) || xalloc(&drho, (size_t)P) ||
            xalloc(&dpsi, (size_t)P) || xalloc(&dinfo, (size_t)nsys) ||
            xalloc(&dchg, 1)) {
            fail(GRMHD_ENOMEM, "device allocation failed");
            break;
        }
        const struct { double* d; const std::vector<double>* v; } ups[] = {
            {dR, &R}, {dS, &S}, {dlam, &lam}, {dQ, &Qs}, {dT, &Ts}, {dbv, &bval}, {dcs, &cs}, {dsn, &sn}};
        bool ok = true;
        for (const auto& u : ups)
            ok = ok && cudaMemcpyAsync(u.d, u.v->data(), u.v->size() * sizeof(double), cudaMemcpyHostToDevice, s) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(dend, endr.data(), endr.size() * sizeof(int), cudaMemcpyHostToDevice, s) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(drho, rho_host, (size_t)P * sizeof(double), cudaMemcpyHostToDevice, s) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(dpsi, psi_host, (size_t)P * sizeof(double), cudaMemcpyHostToDevice, s) == cudaSuccess;
        ok = ok && cudaMemsetAsync(dinfo, 0, sizeof(int) * nsys, s) == cudaSuccess;
        if (!ok) { fail(GRMHD_ECUDA, "upload failed"); break; }
        XDev x;
        x.E = o.E; x.Nr = o.Nr; x.Nt = Nt; x.Np = o.Np; x.n = n; x.nmodes = nmodes; x.nr = nr;
        x.cs = dcs; x.sn = dsn; x.bval = dbv; x.end = dend;
        k_xcts_radial_inverse<<<(unsigned)nsys, 256, 0, s>>>(x, dR, dS, dlam, dA, dinfo);
        if (cudaGetLastError() != cudaSuccess) { fail(GRMHD_ECUDA, "radial inverse launch"); break; }
        std::vector<int> info(nsys);
        if (cudaMemcpyAsync(info.data(), dinfo, sizeof(int) * nsys, cudaMemcpyDeviceToHost, s) ||
            cudaStreamSynchronize(s)) { fail(GRMHD_ECUDA, "factorisation"); break; }
        for (int q = 0; q < nsys; q++)
            if (info[q] != 0) { fail(GRMHD_EINVAL, "singular boundary-value problem (zero pivot)"); break; }
        if (st) break;
        const double setup_ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_setup0).count();
        if (cudaEventCreate(&e1) || cudaEventCreate(&e2)) { fail(GRMHD_ECUDA, "events"); break; }
        cudaEventRecord(e1, s);
        const long long nt_total = (long long)nmodes * 2 * n;
        long long nbt = (nt_total + 255) / 256;
        if (nbt > 152LL * 16) nbt = 152LL * 16;
        // the back substitution keeps one radial vector of nr values in shared memory
        if ((size_t)2 * nr * sizeof(double) > 200 * 1024) {
            fail(GRMHD_EUNSUPPORTED, "more than 12,800 radial nodes");
            break;
        }
        const size_t sm_solve = (size_t)2 * nr * sizeof(double);
        if (sm_solve > 48 * 1024 &&
            cudaFuncSetAttribute(k_xcts_schur_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_solve)) {
            fail(GRMHD_ECUDA, "back substitution shared memory");
            break;
        }
        int done = 0;
        for (int it = 0; it < iters; it++) {
            long long nb = ((long long)n * nmodes + 255) / 256;
            if (nb > 152LL * 16) nb = 152LL * 16;
            k_xcts_forward<<<(unsigned)nb, 256, 0, s>>>(x, drho, dpsi, dB);
            k_xcts_theta<<<(unsigned)nbt, 256, 0, s>>>(x, dQ, dB, dG, 1);
            k_xcts_schur_solve<<<(unsigned)(2 * nmodes), 256, sm_solve, s>>>(x, dA, dT, dS, dG);
            k_xcts_theta<<<(unsigned)nbt, 256, 0, s>>>(x, dQ, dG, dB, 0);
            if (cudaGetLastError() != cudaSuccess) { fail(GRMHD_ECUDA, "iteration launch"); break; }
            unsigned long long z = 0;
            if (cudaMemcpyAsync(dchg, &z, sizeof(z), cudaMemcpyHostToDevice, s)) { fail(GRMHD_ECUDA, "reset"); break; }
            nb = (P + 255) / 256;
            if (nb > 152LL * 16) nb = 152LL * 16;
            k_xcts_inverse<<<(unsigned)nb, 256, 0, s>>>(x, dB, dpsi, dchg);
            if (cudaGetLastError() != cudaSuccess) { fail(GRMHD_ECUDA, "inverse transform launch"); break; }
            unsigned long long cb = 0;
            if (cudaMemcpyAsync(&cb, dchg, sizeof(cb), cudaMemcpyDeviceToHost, s) || cudaStreamSynchronize(s)) {
                fail(GRMHD_ECUDA, "iteration");
                break;
            }
            double c;
            memcpy(&c, &cb, sizeof(c));
            if (changes) changes[it] = c;
            done = it + 1;
            if (!std::isfinite(c)) { fail(GRMHD_ENAN, "the fixed point diverged (non-finite psi)"); break; }
            if (tol > 0.0 && c < tol) break;
        }
        if (st) break;
        cudaEventRecord(e2, s);
        if (cudaMemcpyAsync(psi_host, dpsi, (size_t)P * sizeof(double), cudaMemcpyDeviceToHost, s) ||
            cudaStreamSynchronize(s)) { fail(GRMHD_ECUDA, "download"); break; }
        if (stats) {
            float t2 = 0.f;
            cudaEventElapsedTime(&t2, e1, e2);
            stats[0] = setup_ms;
            stats[1] = done ? t2 / done : 0.0;
            stats[2] = done;
        }
    } while (false);
    cudaStreamSynchronize(s);
    if (e1) cudaEventDestroy(e1);
    if (e2) cudaEventDestroy(e2);
    void* bufs[] = {dR, dS, dlam, dQ, dT, dbv, dcs, dsn, dA, dB, dG, drho, dpsi, dinfo, dend, dchg};
    for (void* b : bufs)
        if (b) cudaFree(b);
    return st;
}

}  // namespace gk
