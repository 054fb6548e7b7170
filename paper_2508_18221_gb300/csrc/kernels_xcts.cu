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
// GPU work: one kernel assembles every L_m densely (column-major, one thread per entry); the
// LU factorisation (once) and the triangular solves (every iteration) are cuSOLVER's
// dgetrf / dgetrs, opened at run time (this step runs once before the time stepping and
// has no other dense solver here); per iteration one kernel forms the source and the
// forward real Fourier transform in phi, and one the inverse transform with the change
// max |psi_{k+1} - psi_k| (block maxima, then one atomic per block).  The modes' LU calls
// are independent and latency-bound, so they are spread over up to 8 side streams.
#include <cuda_runtime.h>
#include <cusolverDn.h>
#include <dlfcn.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "grmhd_internal.h"

namespace gk {

namespace {

struct XDev {
    int E, Nr, Nt, Np, n, nmodes;
    const double* Dr;     // [E][Nr][Nr]
    const double* Drr;    // [E][Nr][Nr]
    const double* D1;     // [2][Nt][Nt] parity +1, -1
    const double* D2;     // [2][Nt][Nt]
    const double* r;      // [E][Nr]
    const double* th;     // [Nt]
    const double* cs;     // [nmodes][Np] cos(2 pi m l / Np)
    const double* sn;     // [nmodes][Np] sin(2 pi m l / Np)
    double M, r_min, r_max;
};

// 0 for a PDE row, 1 for a boundary / interface row; g = its boundary value (phi mode 0)
__device__ __forceinline__ int end_row(const XDev& x, int e, int i, double* g) {
    *g = 0.0;
    if (i == 0) {
        if (e == 0) *g = -x.M / (2.0 * x.r_min * x.r_min);
        return 1;
    }
    if (i == x.Nr - 1) {
        if (e == x.E - 1) *g = 1.0;
        return 1;
    }
    return 0;
}

__global__ void k_xcts_assemble(XDev x, double* __restrict__ L) {
    const long long n = x.n, nn = n * n, total = nn * x.nmodes;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(idx / nn);
        const long long rem = idx - (long long)m * nn;
        const int col = (int)(rem / n), row = (int)(rem - (long long)col * n);
        const int k = row % x.Nt, i = (row / x.Nt) % x.Nr, e = row / (x.Nt * x.Nr);
        const int k2 = col % x.Nt, i2 = (col / x.Nt) % x.Nr, e2 = col / (x.Nt * x.Nr);
        const int s = m & 1;
        const double* Dre = x.Dr + (size_t)e * x.Nr * x.Nr;
        double v = 0.0, g;
        if (!end_row(x, e, i, &g)) {
            if (e2 == e) {
                const double r = x.r[e * x.Nr + i];
                if (k2 == k) v += x.Drr[((size_t)e * x.Nr + i) * x.Nr + i2] + 2.0 / r * Dre[i * x.Nr + i2];
                if (i2 == i) {
                    const double st = sin(x.th[k]), ct = cos(x.th[k]);
                    const double mm = (2 * m == x.Np) ? 0.0 : (double)m * m;
                    double a = x.D2[((size_t)s * x.Nt + k) * x.Nt + k2] + ct / st * x.D1[((size_t)s * x.Nt + k) * x.Nt + k2];
                    if (k2 == k) a -= mm / (st * st);
                    v += a / (r * r);
                }
            }
        } else if (k2 == k) {
            if (i == 0) {
                if (e2 == e) v += Dre[i2];
                if (e > 0 && e2 == e - 1) v -= x.Dr[((size_t)(e - 1) * x.Nr + x.Nr - 1) * x.Nr + i2];
            } else if (e == x.E - 1) {
                if (e2 == e) v += (i2 == i ? 1.0 : 0.0) + x.r_max * Dre[(x.Nr - 1) * x.Nr + i2];
            } else {
                if (e2 == e && i2 == i) v += 1.0;
                if (e2 == e + 1 && i2 == 0) v -= 1.0;
            }
        }
        L[idx] = v;
    }
}

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
        const int i = (q / x.Nt) % x.Nr, e = q / (x.Nt * x.Nr);
        double a = 0.0, b = 0.0, g;
        if (end_row(x, e, i, &g)) {
            a = m == 0 ? g : 0.0;
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

// cuSOLVER, opened at run time so that the library itself does not depend on it
struct Solver {
    void* lib = nullptr;
    decltype(&cusolverDnCreate) create = nullptr;
    decltype(&cusolverDnDestroy) destroy = nullptr;
    decltype(&cusolverDnSetStream) set_stream = nullptr;
    decltype(&cusolverDnDgetrf_bufferSize) getrf_ws = nullptr;
    decltype(&cusolverDnDgetrf) getrf = nullptr;
    decltype(&cusolverDnDgetrs) getrs = nullptr;
};

bool open_solver(Solver* s) {
    const char* names[] = {"libcusolver.so.12", "libcusolver.so", "/usr/local/cuda/lib64/libcusolver.so.12",
                           "/usr/local/cuda/lib64/libcusolver.so"};
    for (const char* nm : names) {
        s->lib = dlopen(nm, RTLD_NOW | RTLD_LOCAL);
        if (s->lib) break;
    }
    if (!s->lib) return false;
    s->create = (decltype(s->create))dlsym(s->lib, "cusolverDnCreate");
    s->destroy = (decltype(s->destroy))dlsym(s->lib, "cusolverDnDestroy");
    s->set_stream = (decltype(s->set_stream))dlsym(s->lib, "cusolverDnSetStream");
    s->getrf_ws = (decltype(s->getrf_ws))dlsym(s->lib, "cusolverDnDgetrf_bufferSize");
    s->getrf = (decltype(s->getrf))dlsym(s->lib, "cusolverDnDgetrf");
    s->getrs = (decltype(s->getrs))dlsym(s->lib, "cusolverDnDgetrs");
    return s->create && s->destroy && s->set_stream && s->getrf_ws && s->getrf && s->getrs;
}

template <class T>
cudaError_t xalloc(T** p, size_t n) { return cudaMalloc((void**)p, n * sizeof(T) + 16); }

}  // namespace

int xcts_solve(const XctsOps& o, const double* rho_host, double* psi_host, int iters, double tol,
               double* changes, double* stats, cudaStream_t s, char* msg, size_t msglen) {
    const int n = o.E * o.Nr * o.Nt, nmodes = o.Np / 2 + 1;
    const long long P = (long long)n * o.Np;
    const size_t nn = (size_t)n * n;
    Solver sv;
    if (!open_solver(&sv)) {
        const char* why = dlerror();
        snprintf(msg, msglen, "cuSOLVER (libcusolver.so.12) could not be opened: %s", why ? why : "missing symbol");
        return GRMHD_EUNSUPPORTED;
    }
    std::vector<double> cs((size_t)nmodes * o.Np), sn((size_t)nmodes * o.Np);
    for (int m = 0; m < nmodes; m++)
        for (int l = 0; l < o.Np; l++) {
            const double a = 2.0 * M_PI * ((long long)m * l % o.Np) / o.Np;
            cs[(size_t)m * o.Np + l] = std::cos(a);
            sn[(size_t)m * o.Np + l] = std::sin(a);
        }
    double *dDr = nullptr, *dDrr = nullptr, *dD1 = nullptr, *dD2 = nullptr, *dr = nullptr, *dth = nullptr,
           *dcs = nullptr, *dsn = nullptr, *dL = nullptr, *dB = nullptr, *drho = nullptr, *dpsi = nullptr;
    int *dpiv = nullptr, *dinfo = nullptr;
    unsigned long long* dchg = nullptr;
    // the modes' factorisations and triangular solves are independent: they run on NS side
    // streams (one cuSOLVER handle and LU workspace each), forked from and joined to s
    const int NS = nmodes < 8 ? nmodes : 8;
    cudaStream_t ss[8] = {};
    cusolverDnHandle_t hs[8] = {};
    double* ws[8] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[8] = {};
    int st = GRMHD_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
    auto fail = [&](int code, const char* what) {
        if (st == GRMHD_OK) {
            st = code;
            snprintf(msg, msglen, "XCTS solve: %s", what);
        }
        return code;
    };
    do {
        if (xalloc(&dDr, o.Dr.size()) || xalloc(&dDrr, o.Drr.size()) || xalloc(&dD1, o.D1.size()) ||
            xalloc(&dD2, o.D2.size()) || xalloc(&dr, o.r.size()) || xalloc(&dth, o.th.size()) ||
            xalloc(&dcs, cs.size()) || xalloc(&dsn, sn.size()) || xalloc(&dL, nn * nmodes) ||
            xalloc(&dB, (size_t)2 * n * nmodes) || xalloc(&drho, (size_t)P) || xalloc(&dpsi, (size_t)P) ||
            xalloc(&dpiv, (size_t)n * nmodes) || xalloc(&dinfo, (size_t)nmodes) || xalloc(&dchg, 1)) {
            fail(GRMHD_ENOMEM, "device allocation failed");
            break;
        }
        const struct { double* d; const std::vector<double>* v; } ups[] = {
            {dDr, &o.Dr}, {dDrr, &o.Drr}, {dD1, &o.D1}, {dD2, &o.D2}, {dr, &o.r}, {dth, &o.th}, {dcs, &cs}, {dsn, &sn}};
        bool ok = true;
        for (const auto& u : ups)
            ok = ok && cudaMemcpyAsync(u.d, u.v->data(), u.v->size() * sizeof(double), cudaMemcpyHostToDevice, s) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(drho, rho_host, (size_t)P * sizeof(double), cudaMemcpyHostToDevice, s) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(dpsi, psi_host, (size_t)P * sizeof(double), cudaMemcpyHostToDevice, s) == cudaSuccess;
        if (!ok) { fail(GRMHD_ECUDA, "upload failed"); break; }
        XDev x;
        x.E = o.E; x.Nr = o.Nr; x.Nt = o.Nt; x.Np = o.Np; x.n = n; x.nmodes = nmodes;
        x.Dr = dDr; x.Drr = dDrr; x.D1 = dD1; x.D2 = dD2; x.r = dr; x.th = dth; x.cs = dcs; x.sn = dsn;
        x.M = o.M; x.r_min = o.r_min; x.r_max = o.r_max;
        if (cudaEventCreate(&e0) || cudaEventCreate(&e1) || cudaEventCreate(&e2)) { fail(GRMHD_ECUDA, "events"); break; }
        cudaEventRecord(e0, s);
        {
            long long nb = ((long long)nn * nmodes + 255) / 256;
            if (nb > 152LL * 32) nb = 152LL * 32;
            k_xcts_assemble<<<(unsigned)nb, 256, 0, s>>>(x, dL);
            if (cudaGetLastError() != cudaSuccess) { fail(GRMHD_ECUDA, "assembly launch"); break; }
        }
        if (cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming)) { fail(GRMHD_ECUDA, "events"); break; }
        for (int j = 0; j < NS && st == GRMHD_OK; j++)
            if (cudaStreamCreateWithFlags(&ss[j], cudaStreamNonBlocking) ||
                cudaEventCreateWithFlags(&ev_join[j], cudaEventDisableTiming) ||
                sv.create(&hs[j]) != CUSOLVER_STATUS_SUCCESS || sv.set_stream(hs[j], ss[j]) != CUSOLVER_STATUS_SUCCESS)
                fail(GRMHD_ECUDA, "cuSOLVER handles / side streams");
        if (st) break;
        int lwork = 0;
        if (sv.getrf_ws(hs[0], n, n, dL, n, &lwork) != CUSOLVER_STATUS_SUCCESS) { fail(GRMHD_ECUDA, "LU workspace size"); break; }
        for (int j = 0; j < NS && st == GRMHD_OK; j++)
            if (xalloc(&ws[j], (size_t)lwork + 1)) fail(GRMHD_ENOMEM, "LU workspace");
        if (st) break;
        auto fork = [&]() {
            cudaEventRecord(ev_fork, s);
            for (int j = 0; j < NS; j++) cudaStreamWaitEvent(ss[j], ev_fork, 0);
        };
        auto join = [&]() {
            for (int j = 0; j < NS; j++) {
                cudaEventRecord(ev_join[j], ss[j]);
                cudaStreamWaitEvent(s, ev_join[j], 0);
            }
        };
        fork();
        for (int m = 0; m < nmodes && st == GRMHD_OK; m++)
            if (sv.getrf(hs[m % NS], n, n, dL + nn * m, n, ws[m % NS], dpiv + (size_t)n * m, dinfo + m) !=
                CUSOLVER_STATUS_SUCCESS)
                fail(GRMHD_ECUDA, "dgetrf failed");
        join();
        if (st) break;
        std::vector<int> info(nmodes);
        if (cudaMemcpyAsync(info.data(), dinfo, sizeof(int) * nmodes, cudaMemcpyDeviceToHost, s) ||
            cudaStreamSynchronize(s)) { fail(GRMHD_ECUDA, "factorisation"); break; }
        for (int m = 0; m < nmodes; m++)
            if (info[m] != 0) { fail(GRMHD_EINVAL, "singular boundary-value problem (dgetrf info != 0)"); break; }
        if (st) break;
        cudaEventRecord(e1, s);
        int done = 0;
        for (int it = 0; it < iters; it++) {
            long long nb = ((long long)n * nmodes + 255) / 256;
            if (nb > 152LL * 16) nb = 152LL * 16;
            k_xcts_forward<<<(unsigned)nb, 256, 0, s>>>(x, drho, dpsi, dB);
            if (cudaGetLastError() != cudaSuccess) { fail(GRMHD_ECUDA, "forward transform launch"); break; }
            fork();
            for (int m = 0; m < nmodes && st == GRMHD_OK; m++)
                if (sv.getrs(hs[m % NS], CUBLAS_OP_N, n, 2, dL + nn * m, n, dpiv + (size_t)n * m, dB + (size_t)2 * n * m, n,
                             dinfo + m) != CUSOLVER_STATUS_SUCCESS)
                    fail(GRMHD_ECUDA, "dgetrs failed");
            join();
            if (st) break;
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
            float t1 = 0.f, t2 = 0.f;
            cudaEventElapsedTime(&t1, e0, e1);
            cudaEventElapsedTime(&t2, e1, e2);
            stats[0] = t1;
            stats[1] = done ? t2 / done : 0.0;
            stats[2] = done;
        }
    } while (false);
    cudaStreamSynchronize(s);
    for (int j = 0; j < NS; j++) {
        if (hs[j]) sv.destroy(hs[j]);
        if (ss[j]) cudaStreamDestroy(ss[j]);
        if (ev_join[j]) cudaEventDestroy(ev_join[j]);
        if (ws[j]) cudaFree(ws[j]);
    }
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e2) cudaEventDestroy(e2);
    void* bufs[] = {dDr, dDrr, dD1, dD2, dr, dth, dcs, dsn, dL, dB, drho, dpsi, dpiv, dinfo, dchg};
    for (void* b : bufs)
        if (b) cudaFree(b);
    return st;
}

}  // namespace gk
