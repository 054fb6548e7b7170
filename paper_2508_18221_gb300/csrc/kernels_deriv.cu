// Spectral derivative / filter contractions and small reductions (FP64).
//
// A derivative along direction dir of a field u[E][Nr][Nt][Np] is the 1-D contraction
// (D u)_i = sum_j D_ij u_j along that axis (paper: "The Spectral Derivative Operators";
// the Chebyshev coefficient route and the Fourier (ik) multiplier are the same linear
// maps written as matrices).  r uses the element's CGL matrix scaled by 2/(b-a), theta
// the Chebyshev-Gauss matrix, phi the circulant Fourier matrix stored as one row.
// r_scale == nullptr applies the matrix unscaled (modal filters).
// One thread produces one output node; the matrix sits in shared memory and a warp
// walks consecutive phi nodes, so every source load of the warp is one coalesced
// 256-byte segment and every matrix load is a broadcast.
#include <math.h>

#include "grmhd_internal.h"

namespace gk {

template <int DIR>
__global__ void __launch_bounds__(256) k_deriv(Dims d, const DerivJob* __restrict__ jobs,
                                               const double* __restrict__ mat,
                                               const double* __restrict__ r_scale) {
    extern __shared__ double sD[];
    const int N = DIR == 0 ? d.Nr : (DIR == 1 ? d.Nt : d.Np);
    const int nmat = DIR == 2 ? N : N * N;
    for (int t = threadIdx.x; t < nmat; t += blockDim.x) sD[t] = mat[t];
    __syncthreads();
    const DerivJob job = jobs[blockIdx.y];
    const long long P = d.P;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P;
         p += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        if (DIR == 2) {
            const int l = (int)(p % N);
            const double* line = job.src + (p - l);
            // (D u)_l = sum_j c[(l - j) mod N] u_j
#pragma unroll 4
            for (int j = 0; j < N; j++) {
                int m = l - j;
                m += (m < 0) ? N : 0;
                acc = fma(sD[m], line[j], acc);
            }
        } else {
            const long long stride = DIR == 0 ? d.NtNp : (long long)d.Np;
            const int i = (int)((p / stride) % N);
            const double* col = job.src + (p - (long long)i * stride);
            const double* Drow = sD + i * N;
#pragma unroll 4
            for (int j = 0; j < N; j++) acc = fma(Drow[j], col[(long long)j * stride], acc);
            if (DIR == 0 && r_scale != nullptr) acc *= r_scale[p / d.elem];
        }
        if (job.accumulate) job.dst[p] += acc;
        else job.dst[p] = acc;
    }
}

cudaError_t launch_deriv(int dir, const Dims& d, const DerivJob* jobs_dev, int njobs,
                         const double* mat_dev, const double* r_scale_dev, cudaStream_t s) {
    if (njobs <= 0) return cudaSuccess;
    const int bs = 256;
    long long nb = (d.P + bs - 1) / bs;
    if (nb > 65535LL * 32) nb = 65535LL * 32;
    dim3 grid((unsigned)nb, (unsigned)njobs);
    const int N = dir == 0 ? d.Nr : (dir == 1 ? d.Nt : d.Np);
    size_t sm = (size_t)(dir == 2 ? N : N * N) * sizeof(double);
    if (dir == 0) k_deriv<0><<<grid, bs, sm, s>>>(d, jobs_dev, mat_dev, r_scale_dev);
    else if (dir == 1) k_deriv<1><<<grid, bs, sm, s>>>(d, jobs_dev, mat_dev, r_scale_dev);
    else k_deriv<2><<<grid, bs, sm, s>>>(d, jobs_dev, mat_dev, r_scale_dev);
    return cudaGetLastError();
}

cudaError_t eo_init();
cudaError_t tc_init();

cudaError_t kernels_init() {
    cudaError_t e;
    // dense contractions: theta matrices up to 128 x 128 doubles (128 KB)
    if ((e = cudaFuncSetAttribute(k_deriv<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 64 * 8)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_deriv<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 128 * 8)) != cudaSuccess) return e;
    if ((e = eo_init()) != cudaSuccess) return e;
    if ((e = fx_init()) != cudaSuccess) return e;
    return tc_init();
}

// Replace both copies of each duplicated interface node by their mean.
template <typename T>
__global__ void k_iface_avg(Dims d, T* base, long long fstride, int nfields) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long nif = (long long)(d.E - 1) * d.NtNp;
    if (t >= nif * nfields) return;
    int f = (int)(t / nif);
    long long r = t % nif;
    int e = (int)(r / d.NtNp);
    long long kl = r % d.NtNp;
    if (!d.iface_next[e]) return;  // instance boundary inside a batch group
    T* u = base + f * fstride;
    long long pl = (long long)e * d.elem + (long long)(d.Nr - 1) * d.NtNp + kl;
    long long pr = pl + d.NtNp;
    T m = (T)0.5 * (u[pl] + u[pr]);
    u[pl] = m;
    u[pr] = m;
}

cudaError_t launch_iface_avg(const Dims& d, double* base, long long fstride, int nfields,
                             cudaStream_t s) {
    if (d.E < 2 || nfields <= 0) return cudaSuccess;
    long long n = (long long)(d.E - 1) * d.NtNp * nfields;
    int bs = 256;
    k_iface_avg<double><<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(d, base, fstride, nfields);
    return cudaGetLastError();
}

cudaError_t launch_iface_avg_f(const Dims& d, float* base, long long fstride, int nfields,
                               cudaStream_t s) {
    if (d.E < 2 || nfields <= 0) return cudaSuccess;
    long long n = (long long)(d.E - 1) * d.NtNp * nfields;
    int bs = 256;
    k_iface_avg<float><<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(d, base, fstride, nfields);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- Fourier theta folding
// The theta derivative (or filter) of the double-Fourier extension couples the lines at
// phi and phi + pi: out(phi) = A u(phi) + s B u(phi + pi) with the parity s of the field.
// With the sum p and difference m of the pair, out(phi) = (A + s B)/2 p + (A - s B)/2 m
// and out(phi + pi) = (A + s B)/2 p - (A - s B)/2 m, so the fold writes p and m into two
// halves of N_phi / 2 lines per row (the half for the even operator first: p when s = +1,
// m when s = -1), each half is contracted along theta with one operator (the 1/2 is in the
// operators, so the fold spends one FP64 addition per value and no multiplication: GB300's
// FP64 pipe bounded it), and the unfold adds and subtracts the two results.  Pure
// streaming: one coalesced read and write per value.
template <typename T>
__global__ void k_theta_fold(Dims d, const FoldJob* __restrict__ jobs) {
    const FoldJob jb = jobs[blockIdx.y];
    const T* __restrict__ src = static_cast<const T*>(jb.src);
    T* __restrict__ dst = static_cast<T*>(jb.dst);
    const int h = d.Np / 2;
    const long long half = d.P / 2;
#pragma unroll 4
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < half;
         t += (long long)gridDim.x * blockDim.x) {
        const long long row = t / h;
        const long long i0 = row * d.Np + (t - row * h);
        const T a = src[i0], b = src[i0 + h];
        const T p = a + b, m = a - b;
        dst[t] = jb.parity > 0 ? p : m;
        dst[half + t] = jb.parity > 0 ? m : p;
    }
}

template <typename T>
__global__ void k_theta_unfold(Dims d, const FoldJob* __restrict__ jobs) {
    const FoldJob jb = jobs[blockIdx.y];
    const T* __restrict__ src = static_cast<const T*>(jb.src);
    T* __restrict__ dst = static_cast<T*>(jb.dst);
    const int h = d.Np / 2;
    const long long half = d.P / 2;
#pragma unroll 4
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < half;
         t += (long long)gridDim.x * blockDim.x) {
        const T z0 = src[t], z1 = src[half + t];
        const T zp = jb.parity > 0 ? z0 : z1, zm = jb.parity > 0 ? z1 : z0;
        const long long row = t / h;
        const long long i0 = row * d.Np + (t - row * h);
        if (jb.accumulate) {
            dst[i0] += zp + zm;
            dst[i0 + h] += zp - zm;
        } else {
            dst[i0] = zp + zm;
            dst[i0 + h] = zp - zm;
        }
    }
}

// about four elements per thread (the loops above are unrolled by four: their loads are
// independent, so four are in flight per thread)
static dim3 fold_grid(const Dims& d, int njobs) {
    long long nb = (d.P / 2 + 1023) / 1024;
    if (nb > 152LL * 16) nb = 152LL * 16;
    return dim3((unsigned)nb, (unsigned)njobs);
}

cudaError_t launch_theta_fold(const Dims& d, const FoldJob* jobs, int njobs, int fp32, cudaStream_t s) {
    if (njobs <= 0 || d.P <= 0) return cudaSuccess;
    if (d.Np % 2) return cudaErrorInvalidValue;
    if (fp32) k_theta_fold<float><<<fold_grid(d, njobs), 256, 0, s>>>(d, jobs);
    else k_theta_fold<double><<<fold_grid(d, njobs), 256, 0, s>>>(d, jobs);
    return cudaGetLastError();
}

cudaError_t launch_theta_unfold(const Dims& d, const FoldJob* jobs, int njobs, int fp32, cudaStream_t s) {
    if (njobs <= 0 || d.P <= 0) return cudaSuccess;
    if (d.Np % 2) return cudaErrorInvalidValue;
    if (fp32) k_theta_unfold<float><<<fold_grid(d, njobs), 256, 0, s>>>(d, jobs);
    else k_theta_unfold<double><<<fold_grid(d, njobs), 256, 0, s>>>(d, jobs);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- CFL time step
// lambda = |beta|_gamma + max(alpha, sqrt(2 alpha)); max over nodes by atomicMax on the
// bit pattern (order-preserving for non-negative doubles); dt = cfl hmin / lambda_max.
__global__ void k_cfl_lam(Dims d, const double* __restrict__ U, unsigned long long* bits) {
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long P = d.P;
    double lam = 0.0;
    int inst = -1;
    if (p < P) {
        inst = d.elem_inst[p / d.elem];
        double e4 = exp(4.0 * U[V_PHI * P + p]);
        double b[3] = {U[V_BETA * P + p], U[(V_BETA + 1) * P + p], U[(V_BETA + 2) * P + p]};
        const int sidx[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
        double bb = 0.0;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) bb += b[i] * b[j] * U[(V_GT + sidx[i][j]) * P + p];
        double al = U[V_ALPHA * P + p];
        lam = sqrt(e4 * bb) + fmax(al, sqrt(2.0 * al));
        if (!(lam >= 0.0)) lam = INFINITY;
    }
    // warp maximum when the whole warp belongs to one instance, else one atomic per node
    const int i0 = __shfl_sync(0xffffffffu, inst, 0);
    if (__all_sync(0xffffffffu, inst == i0)) {
        for (int o = 16; o > 0; o >>= 1) lam = fmax(lam, __shfl_xor_sync(0xffffffffu, lam, o));
        if ((threadIdx.x & 31) == 0 && i0 >= 0) atomicMax(&bits[i0], (unsigned long long)__double_as_longlong(lam));
    } else if (inst >= 0) {
        atomicMax(&bits[inst], (unsigned long long)__double_as_longlong(lam));
    }
}

__global__ void k_cfl_dt(int n_inst, const unsigned long long* bits, const double* hmin, double cfl,
                         double* dt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_inst) return;
    double lam = __longlong_as_double((long long)bits[i]);
    dt[i] = cfl * hmin[i] / lam;
}

cudaError_t launch_cfl(const Dims& d, int n_inst, const double* U, const double* hmin_dev, double cfl,
                       double* dt_dev, unsigned long long* bits, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(unsigned long long) * n_inst, s);
    if (e != cudaSuccess) return e;
    int bs = 256;
    k_cfl_lam<<<(unsigned)((d.P + bs - 1) / bs), bs, 0, s>>>(d, U, bits);
    k_cfl_dt<<<(n_inst + 127) / 128, 128, 0, s>>>(n_inst, bits, hmin_dev, cfl, dt_dev);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- diagnostics
// out[0] += w D~, out[1] += w rho s sqrt(gamma), out[2] = max |divB| (bits)
__global__ void k_diag(Dims d, PhysParams pp, const double* __restrict__ U,
                       const double* __restrict__ prim, const double* __restrict__ wq,
                       const double* __restrict__ divB, const double* __restrict__ ham, double* out) {
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long P = d.P;
    double m = 0.0, s = 0.0, db = 0.0, hm = 0.0, h2 = 0.0, ws = 0.0;
    if (p < P) {
        double e4 = exp(4.0 * U[V_PHI * P + p]);
        const int sidx[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
        double g[3][3];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) g[i][j] = e4 * U[(V_GT + sidx[i][j]) * P + p];
        double det = g[0][0] * (g[1][1] * g[2][2] - g[1][2] * g[2][1]) -
                     g[0][1] * (g[1][0] * g[2][2] - g[1][2] * g[2][0]) +
                     g[0][2] * (g[1][0] * g[2][1] - g[1][1] * g[2][0]);
        double rho = prim[p], pr = prim[5 * P + p];
        m = wq[p] * U[V_D * P + p];
        s = wq[p] * rho * (log(pr / pow(rho, pp.gam)) / (pp.gam - 1.0)) * sqrt(det);
        db = fabs(divB[p]);
        if (ham) {
            hm = fabs(ham[p]);
            h2 = wq[p] * ham[p] * ham[p];
            ws = wq[p];
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        m += __shfl_xor_sync(0xffffffffu, m, o);
        s += __shfl_xor_sync(0xffffffffu, s, o);
        db = fmax(db, __shfl_xor_sync(0xffffffffu, db, o));
        hm = fmax(hm, __shfl_xor_sync(0xffffffffu, hm, o));
        h2 += __shfl_xor_sync(0xffffffffu, h2, o);
        ws += __shfl_xor_sync(0xffffffffu, ws, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], m);
        atomicAdd(&out[1], s);
        atomicMax(reinterpret_cast<unsigned long long*>(&out[2]),
                  (unsigned long long)__double_as_longlong(db));
        if (ham) {
            atomicMax(reinterpret_cast<unsigned long long*>(&out[5]),
                      (unsigned long long)__double_as_longlong(hm));
            atomicAdd(&out[6], h2);
            atomicAdd(&out[7], ws);
        }
    }
}

cudaError_t launch_diag(const Dims& d, const PhysParams& pp, const double* U,
                        const double* prim, const double* wq, const double* divB,
                        double* out_dev, cudaStream_t s, const double* ham) {
    int bs = 256;
    k_diag<<<(unsigned)((d.P + bs - 1) / bs), bs, 0, s>>>(d, pp, U, prim, wq, divB, ham, out_dev);
    return cudaGetLastError();
}

__global__ void k_nan(long long n, const double* __restrict__ U, int* flag) {
    int bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        bad |= !isfinite(U[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

cudaError_t launch_nan_check(long long n, const double* U, int* flag, cudaStream_t s) {
    int bs = 256;
    long long nb = (n + bs - 1) / bs;
    if (nb > 4096) nb = 4096;
    k_nan<<<(unsigned)nb, bs, 0, s>>>(n, U, flag);
    return cudaGetLastError();
}

}  // namespace gk
