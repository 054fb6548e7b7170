// Reflection-split contractions (FP64): the same linear maps as k_deriv with half the
// fused multiply-adds.
//
// Every 1-D operator of the grid either commutes (modal filters, sign +1) or
// anticommutes (first derivatives, sign -1) with the reflection of its node set:
// x_j -> -x_j on the Chebyshev nodes (j <-> N-1-j) and phi_j -> -phi_j on the Fourier
// nodes (j <-> N-j, fixed points j = 0 and N/2).  Writing a line u as its even and odd
// parts over the index pairs (j, j'),  s_j = u_j + u_j',  a_j = u_j - u_j',  gives for an
// output pair (i, i')
//     out_i  = E s + O a + C u_f,        out_i' = sign (E s - O a + C u_f),
// with E = (D_ij + D_ij')/2, O = (D_ij - D_ij')/2 and C the columns of the fixed points,
// so a pair of outputs costs N fused multiply-adds instead of 2N.  One thread owns one
// line: it loads the N values into registers, forms s and a once, and writes its N
// outputs; the split matrices sit in shared memory and every matrix read of a warp is a
// broadcast.  FP64 throughput, not memory, bounds this kernel on GB300 (1.2 TFLOP/s vs
// 6.8 TB/s), so the strided per-thread line accesses cost nothing measurable.
#include "grmhd_internal.h"

namespace gk {

// KIND 0: Chebyshev (pairs j <-> N-1-j, middle node fixed for odd N)
// KIND 1: Fourier   (pairs j <-> N-j for j = 1..N/2-1, fixed 0 and N/2; N even)
template <int KIND, int N>
struct Split {
    static constexpr int NP = KIND == 0 ? N / 2 : N / 2 - 1;
    static constexpr int NF = KIND == 0 ? N % 2 : 2;
    static constexpr int SIZE = 2 * NP * NP + 2 * NP * NF + NF * NF;
    __device__ static constexpr int pair_lo(int ip) { return KIND == 0 ? ip : ip + 1; }
    __device__ static constexpr int pair_hi(int ip) { return N - 1 - ip; }
    __device__ static constexpr int fixed(int f) { return KIND == 0 ? N / 2 : (f == 0 ? 0 : N / 2); }
};

template <int DIR, int KIND, int N>
__global__ void __launch_bounds__(128) k_deriv_eo(Dims d, const DerivJob* __restrict__ jobs,
                                                  const double* __restrict__ op, int sign,
                                                  const double* __restrict__ r_scale) {
    using S = Split<KIND, N>;
    constexpr int NP = S::NP, NF = S::NF;
    extern __shared__ double sm[];
    for (int t = threadIdx.x; t < S::SIZE; t += blockDim.x) sm[t] = op[t];
    __syncthreads();
    const double* E = sm;
    const double* O = E + NP * NP;
    const double* C = O + NP * NP;        // [NP][NF]
    const double* F = C + NP * NF;        // [NF][NP]
    const double* G = F + NF * NP;        // [NF][NF]
    const DerivJob job = jobs[blockIdx.y];

    long long nlines, stride;
    if (DIR == 0) { nlines = (long long)d.E * d.NtNp; stride = d.NtNp; }
    else if (DIR == 1) { nlines = (long long)d.E * d.Nr * d.Np; stride = d.Np; }
    else { nlines = d.P / N; stride = 1; }

    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nlines;
         t += (long long)gridDim.x * blockDim.x) {
        long long base;
        double scale = 1.0;
        if (DIR == 0) {
            long long e = t / d.NtNp;
            base = e * d.elem + (t - e * d.NtNp);
            if (r_scale) scale = r_scale[e];
        } else if (DIR == 1) {
            long long eil = t / d.Np;
            base = eil * d.NtNp + (t - eil * d.Np);
        } else {
            base = t * N;
        }
        const double* src = job.src + base;
        double s[NP > 0 ? NP : 1], a[NP > 0 ? NP : 1], uf[NF > 0 ? NF : 1];
#pragma unroll
        for (int j = 0; j < NP; j++) {
            double lo = src[(long long)S::pair_lo(j) * stride];
            double hi = src[(long long)S::pair_hi(j) * stride];
            s[j] = lo + hi;
            a[j] = lo - hi;
        }
#pragma unroll
        for (int f = 0; f < NF; f++) uf[f] = src[(long long)S::fixed(f) * stride];
        double* dst = job.dst + base;
        for (int ip = 0; ip < NP; ip++) {
            const double* Er = E + ip * NP;
            const double* Or = O + ip * NP;
            double A = 0.0, B = 0.0, Cc = 0.0;
#pragma unroll
            for (int j = 0; j < NP; j++) {
                A = fma(Er[j], s[j], A);
                B = fma(Or[j], a[j], B);
            }
#pragma unroll
            for (int f = 0; f < NF; f++) Cc = fma(C[ip * NF + f], uf[f], Cc);
            double o1 = (A + B + Cc) * scale;
            double o2 = sign * (A - B + Cc) * scale;
            long long i1 = (long long)S::pair_lo(ip) * stride, i2 = (long long)S::pair_hi(ip) * stride;
            if (job.accumulate) { dst[i1] += o1; dst[i2] += o2; }
            else { dst[i1] = o1; dst[i2] = o2; }
        }
#pragma unroll
        for (int f = 0; f < NF; f++) {
            double acc = 0.0;
#pragma unroll
            for (int j = 0; j < NP; j++) acc = fma(F[f * NP + j], sign < 0 ? a[j] : s[j], acc);
#pragma unroll
            for (int g = 0; g < NF; g++) acc = fma(G[f * NF + g], uf[g], acc);
            acc *= scale;
            long long i1 = (long long)S::fixed(f) * stride;
            if (job.accumulate) dst[i1] += acc;
            else dst[i1] = acc;
        }
    }
}

template <int DIR, int KIND, int N>
static cudaError_t launch_one(const Dims& d, const DerivJob* jobs, int njobs, const double* op,
                              int sign, const double* r_scale, cudaStream_t s) {
    using S = Split<KIND, N>;
    long long nlines = DIR == 0 ? (long long)d.E * d.NtNp : (DIR == 1 ? (long long)d.E * d.Nr * d.Np : d.P / N);
    const int bs = 128;
    long long nb = (nlines + bs - 1) / bs;
    if (nb > 65535LL * 16) nb = 65535LL * 16;
    size_t sm = (size_t)S::SIZE * sizeof(double);
    k_deriv_eo<DIR, KIND, N><<<dim3((unsigned)nb, (unsigned)njobs), bs, sm, s>>>(d, jobs, op, sign, r_scale);
    return cudaGetLastError();
}

#define CHEB_CASE(n) case n: return launch_one<DIR, 0, n>(d, jobs, njobs, op, sign, r_scale, s);
#define FOUR_CASE(n) case n: return launch_one<DIR, 1, n>(d, jobs, njobs, op, sign, r_scale, s);

template <int DIR>
static cudaError_t dispatch(int N, const Dims& d, const DerivJob* jobs, int njobs, const double* op,
                            int sign, const double* r_scale, cudaStream_t s) {
    if (DIR < 2) {
        switch (N) {
            CHEB_CASE(4) CHEB_CASE(5) CHEB_CASE(6) CHEB_CASE(7) CHEB_CASE(8) CHEB_CASE(9)
            CHEB_CASE(10) CHEB_CASE(11) CHEB_CASE(12) CHEB_CASE(13) CHEB_CASE(14) CHEB_CASE(15)
            CHEB_CASE(16) CHEB_CASE(20) CHEB_CASE(24) CHEB_CASE(32) CHEB_CASE(40) CHEB_CASE(48)
            CHEB_CASE(64)
            default: return cudaErrorNotSupported;
        }
    } else {
        switch (N) {
            FOUR_CASE(4) FOUR_CASE(6) FOUR_CASE(8) FOUR_CASE(10) FOUR_CASE(12) FOUR_CASE(16)
            FOUR_CASE(20) FOUR_CASE(24) FOUR_CASE(32) FOUR_CASE(48) FOUR_CASE(64) FOUR_CASE(128)
            default: return cudaErrorNotSupported;
        }
    }
}

cudaError_t eo_init() {
    // the only instance above the default 48 KB: Fourier N = 128 (65.5 KB)
    return cudaFuncSetAttribute(k_deriv_eo<2, 1, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(Split<1, 128>::SIZE * sizeof(double)));
}

bool eo_supported(int dir, int N) {
    static const int cheb[] = {4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 20, 24, 32, 40, 48, 64};
    static const int four[] = {4, 6, 8, 10, 12, 16, 20, 24, 32, 48, 64, 128};
    if (dir < 2) {
        for (int v : cheb) if (v == N) return true;
    } else {
        for (int v : four) if (v == N) return true;
    }
    return false;
}

cudaError_t launch_deriv_eo(int dir, const Dims& d, const DerivJob* jobs, int njobs,
                            const double* op_split, int sign, const double* r_scale,
                            cudaStream_t s) {
    if (njobs <= 0) return cudaSuccess;
    if (dir == 0) return dispatch<0>(d.Nr, d, jobs, njobs, op_split, sign, r_scale, s);
    if (dir == 1) return dispatch<1>(d.Nt, d, jobs, njobs, op_split, sign, nullptr, s);
    return dispatch<2>(d.Np, d, jobs, njobs, op_split, sign, nullptr, s);
}

}  // namespace gk
