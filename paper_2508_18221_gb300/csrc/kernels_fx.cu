// FP64-accurate spectral contractions on the BF16 tensor cores (tcgen05, sm_103a).
//
// out[line][i] = sum_j D[i][j] u[line][j] in double precision, computed with the
// error-free splitting of Ozaki, Ogita, Oishi & Rump (Numer. Algorithms 59, 2012):
//   * every line of u gets one common exponent (its largest), every row of D its own;
//     relative to it each value is a signed 54-bit fixed-point integer, written as seven
//     balanced base-256 digits d_1..d_7 in [-128, 127] (most significant first);
//   * a digit fits a BF16 exactly and a product of two digits (|.| <= 2^14) fits an FP32
//     exactly, so the tensor core forms sum_j c_l(i,j) d_q(j) without rounding as long as
//     the running sum stays below 2^24 (true for K <= 64 and the groups below);
//   * the 28 digit pairs with q + l <= 8 are kept; those with q + l = 2, 3, 4, 5
//     accumulate in four separate TMEM accumulators (exact), those with q + l = 6..8 in
//     a fifth (its FP32 rounding lies 2^-56 below the leading term);
//   * the epilogue adds the five accumulators as a 64-bit integer and builds the IEEE
//     double with integer instructions (no FP64 arithmetic: GB300 runs FP64 at ~2 fused
//     operations per SM clock, integer and FP32 work at 64-128).
// Error: about 2^-53 of sum_j |D_ij| max_j |u_j| (truncated digits, dropped pairs,
// rounding of the fifth accumulator), within the bound of an FP64 dot product.  A line
// holding Inf or NaN yields NaN outputs; values below 2^-1022 (subnormals) enter as zero.
//
// Tile: 128 lines (one per thread and TMEM lane) x K (<= 64 nodes: five accumulators of
// up to 64 columns fill the 512 TMEM columns), processed in K chunks of KC = 16 or 32.
// The operator's seven digit slices for a chunk are prepared on the host in the K-major
// core-matrix layout (8 rows x 16 bytes per core matrix) and fetched with one
// cp.async.bulk; the line digits are formed by the threads from the FP64 bits.  TMEM is
// allocated only after the first chunk's digits are in shared memory, so that a second
// CTA on the SM prepares its tile while the first one multiplies.  Waits are bounded and
// report through *err.
#include <cuda_bf16.h>
#include <stdint.h>

#include "grmhd_internal.h"

namespace gk {

namespace {

constexpr int NDIG = 7;                                      // base-256 digits per operand
constexpr int NACC = 5;                                      // TMEM accumulators
constexpr unsigned long long DIG_BIAS = 0x80808080808080ull;  // 128 in each digit

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // tcgen05 descriptor version
    return d;                // base offset 0, relative LBO, no swizzle
}

// D = F32, A = B = BF16, both K-major; N >> 3 at bit 17, M >> 4 at bit 24
__device__ __forceinline__ uint32_t instr_desc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
    uint32_t done = 0;
    for (int it = 0; it < (1 << 22) && !done; it++)
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(smem_u32(bar)), "r"(phase) : "memory");
    return done != 0;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t id, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                 "l"(da), "l"(db), "r"(id), "r"(acc));
}

// Digit word of one value: Z = X + bias with X = round(2 m 2^(e - EL)) the value as a
// signed fixed-point integer relative to the line exponent EL (|X| <= 2^54; the value is
// X 2^(EL - 1076)); byte b of Z minus 128 is the balanced digit of weight 256^b.
__device__ __forceinline__ unsigned long long digit_word(double u, int EL) {
    const long long bits = __double_as_longlong(u);
    const int e = (int)((bits >> 52) & 0x7FF);
    const unsigned long long m2 = (((unsigned long long)bits & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 1;
    const int sh = EL - e;  // >= 0
    unsigned long long mag = 0;
    if (e != 0) {
        if (sh == 0) mag = m2;
        else if (sh < 60) mag = (m2 + (1ull << (sh - 1))) >> sh;
    }
    const long long x = bits < 0 ? -(long long)mag : (long long)mag;
    return (unsigned long long)(x + (long long)DIG_BIAS);
}

// FP32 value (b - 128) * 2^(-8 (q-1)) of byte b of `w` (byte index sel 0..3): the byte is
// placed in the mantissa of 1.5 * 2^23 and the offset removed by one exact FMA.
template <int Q>
__device__ __forceinline__ float digit_val(uint32_t w, int sel) {
    constexpr float S = Q == 1 ? 1.f : (Q == 2 ? 0x1p-8f : (Q == 3 ? 0x1p-16f : (Q == 4 ? 0x1p-24f : (Q == 5 ? 0x1p-32f : (Q == 6 ? 0x1p-40f : 0x1p-48f)))));
    const float f = __uint_as_float(__byte_perm(w, 0x4B400000u, 0x7640u | (uint32_t)sel));
    return fmaf(f, S, -12583040.f * S);
}

// two BF16 (exact: at most 8 significant bits) packed low = a, high = b
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632u);
}

// R * 2^X as an IEEE double built with integer instructions (|R| < 2^62; ties away)
__device__ __forceinline__ double ldexp_int(long long R, int X) {
    if (R == 0) return 0.0;
    const unsigned long long sgn = R < 0 ? (1ull << 63) : 0ull;
    const unsigned long long a = R < 0 ? (unsigned long long)(-R) : (unsigned long long)R;
    const int p = 63 - __clzll((long long)a);
    unsigned long long mant;
    if (p <= 52) mant = a << (52 - p);
    else { const int sh = p - 52; mant = (a + (1ull << (sh - 1))) >> sh; }
    const int be = p + X + 1023;
    if (be <= 0) return __longlong_as_double((long long)sgn);
    if (be >= 2047) return __longlong_as_double((long long)(sgn | 0x7FF0000000000000ull));
    return __longlong_as_double((long long)(sgn | ((((unsigned long long)(be - 1)) << 52) + mant)));
}

// T = g2 + g3 + g4 + g5 + gf as the integer R = round(T 2^40): g2 is an integer, g3 a
// multiple of 2^-8, g4 of 2^-16, g5 of 2^-24 (all exact, |g_s 2^(8 (s-2))| <= 2^22 for
// K <= 64), gf carries the rounded low-order terms (|gf| < 2^-8).
__device__ __forceinline__ long long combine(float g2, float g3, float g4, float g5, float gf) {
    const float MAG = 12582912.f;  // 1.5 * 2^23: float -> nearest integer for |x| <= 2^22
    const int n2 = __float_as_int(g2 + MAG) - 0x4B400000;
    const int n3 = __float_as_int(fmaf(g3, 256.f, MAG)) - 0x4B400000;
    const int n4 = __float_as_int(fmaf(g4, 65536.f, MAG)) - 0x4B400000;
    const int n5 = __float_as_int(fmaf(g5, 16777216.f, MAG)) - 0x4B400000;
    const float fh = fmaf(gf, 16777216.f, MAG);
    const int nfh = __float_as_int(fh) - 0x4B400000;
    const float flo = fmaf(gf, 16777216.f, -(fh - MAG));  // exact remainder in [-1/2, 1/2]
    const int nlo = __float_as_int(fmaf(flo, 65536.f, MAG)) - 0x4B400000;
    const long long a = ((long long)n2 << 24) + ((long long)n3 << 16) + ((long long)n4 << 8) + (long long)(n5 + nfh);
    return (a << 16) + (long long)nlo;
}

}  // namespace

// Shared memory (bytes): [A digits 7 x 128 x KC x 2 | B digits 7 x Np x KC x 2 |
//                         row exponents Np x 4 | 2 mbarriers | tmem address]
template <int DIR>
__global__ void __launch_bounds__(128) k_contract_fx(Dims d, const DerivJob* __restrict__ jobs,
                                                     const uint8_t* __restrict__ img, long long img_estride,
                                                     int N, int Np, int Kp, int KC, int tmem_cols,
                                                     int* __restrict__ err) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int kcores = KC / 8;
    const uint32_t a_bytes = 128u * KC * 2;
    const uint32_t b_bytes = (uint32_t)Np * KC * 2;
    const uint32_t chunk_bytes = NDIG * b_bytes;
    const int nchunks = Kp / KC;
    uint8_t* sA = sm;
    uint8_t* sB = sm + NDIG * a_bytes;
    int* sF = reinterpret_cast<int*>(sB + chunk_bytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sF + Np);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);
    const DerivJob job = jobs[blockIdx.y];

    // this thread's line
    long long base = 0, stride;
    bool valid;
    const uint8_t* op = img;
    if (DIR == 0) {
        const long long tpe = (d.NtNp + 127) / 128;
        const long long e = blockIdx.x / tpe;
        const long long lt = (blockIdx.x - e * tpe) * 128 + tid;
        valid = lt < d.NtNp;
        base = e * d.elem + lt;
        stride = d.NtNp;
        op = img + e * img_estride;
    } else if (DIR == 1) {
        const long long t = (long long)blockIdx.x * 128 + tid;
        valid = t < (long long)d.E * d.Nr * d.Np;
        const long long eil = t / d.Np;
        base = eil * d.NtNp + (t - eil * d.Np);
        stride = d.Np;
    } else {
        const long long t = (long long)blockIdx.x * 128 + tid;
        valid = t < d.P / N;
        base = t * N;
        stride = 1;
    }
    const double* src = job.src;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    const int* op_exp = reinterpret_cast<const int*>(op + (size_t)nchunks * chunk_bytes);
    for (int n = tid; n < Np; n += 128) sF[n] = op_exp[n];

    // pass 1: the line's largest biased exponent
    int EL = 0;
    if (valid) {
        if (DIR == 2) {
            const double2* p2 = reinterpret_cast<const double2*>(src + base);
            for (int j = 0; j < N / 2; j++) {
                const double2 v = p2[j];
                EL = max(EL, (int)((__double_as_longlong(v.x) >> 52) & 0x7FF));
                EL = max(EL, (int)((__double_as_longlong(v.y) >> 52) & 0x7FF));
            }
        } else {
            const int* hi = reinterpret_cast<const int*>(src + base) + 1;
            for (int j = 0; j < N; j++) EL = max(EL, (hi[2LL * j * stride] >> 20) & 0x7FF);
        }
    }
    const bool line_bad = EL == 0x7FF;
    __syncthreads();  // barrier initialisation visible before the first bulk copy

    uint32_t tmem = 0;
    bool ok = true;
    for (int kc = 0; kc < nchunks; kc++) {
        if (kc > 0 && !mbar_wait(&bars[1], (kc - 1) & 1)) ok = false;
        if (tid == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bars[0])),
                         "r"(chunk_bytes) : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             smem_u32(sB)),
                         "l"(op + (size_t)kc * chunk_bytes), "r"(chunk_bytes), "r"(smem_u32(&bars[0]))
                         : "memory");
        }
        // line digits of this chunk, 8 K values (one 16-byte core-matrix row per digit) at a time
        for (int g8 = 0; g8 < kcores; g8++) {
            const int k0 = kc * KC + g8 * 8;
            uint32_t w[NDIG][4];
#pragma unroll
            for (int h = 0; h < 4; h++) {
                double u0 = 0.0, u1 = 0.0;
                const int k = k0 + 2 * h;
                if (valid) {
                    if (DIR == 2) {
                        if (k < N) {  // N even: pairs never straddle the line end
                            const double2 v = *reinterpret_cast<const double2*>(src + base + k);
                            u0 = v.x;
                            u1 = v.y;
                        }
                    } else {
                        if (k < N) u0 = src[base + (long long)k * stride];
                        if (k + 1 < N) u1 = src[base + (long long)(k + 1) * stride];
                    }
                }
                const unsigned long long z0 = digit_word(u0, EL), z1 = digit_word(u1, EL);
                const uint32_t l0 = (uint32_t)z0, h0 = (uint32_t)(z0 >> 32);
                const uint32_t l1 = (uint32_t)z1, h1 = (uint32_t)(z1 >> 32);
                // digit q (1 = most significant) is byte 7 - q of Z
                w[0][h] = pack_bf16(digit_val<1>(h0, 2), digit_val<1>(h1, 2));
                w[1][h] = pack_bf16(digit_val<2>(h0, 1), digit_val<2>(h1, 1));
                w[2][h] = pack_bf16(digit_val<3>(h0, 0), digit_val<3>(h1, 0));
                w[3][h] = pack_bf16(digit_val<4>(l0, 3), digit_val<4>(l1, 3));
                w[4][h] = pack_bf16(digit_val<5>(l0, 2), digit_val<5>(l1, 2));
                w[5][h] = pack_bf16(digit_val<6>(l0, 1), digit_val<6>(l1, 1));
                w[6][h] = pack_bf16(digit_val<7>(l0, 0), digit_val<7>(l1, 0));
            }
            const uint32_t off = (uint32_t)(((tid >> 3) * kcores + g8) * 128 + (tid & 7) * 16);
#pragma unroll
            for (int q = 0; q < NDIG; q++)
                *reinterpret_cast<uint4*>(sA + q * a_bytes + off) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (kc == 0) {
            // tensor memory only from here on (see the header)
            if (warp == 0) {
                asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                                 smem_u32(tmem_slot)),
                             "r"(tmem_cols));
                asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        tmem = *tmem_slot;
        if (tid == 0) {
            if (mbar_wait(&bars[0], kc & 1)) {
                const uint32_t id = instr_desc_bf16(128, Np);
                const uint32_t lbo = 128u, sbo = (uint32_t)kcores * 128u;
                // digit pairs (q, l), 0-based, s = q + l <= 6 into accumulator min(s, 4);
                // within the folded accumulator the smallest terms come first
                for (int s = NDIG - 1; s >= 0; s--) {
                    const int g = s < NACC - 1 ? s : NACC - 1;
                    for (int q = 0; q <= s; q++) {
                        const int l = s - q;
                        const bool first = kc == 0 && q == 0 && (s < NACC - 1 || s == NDIG - 1);
                        for (int c = 0; c < KC / 16; c++) {
                            const uint64_t da = smem_desc(smem_u32(sA + q * a_bytes) + c * 256, lbo, sbo);
                            const uint64_t db = smem_desc(smem_u32(sB + l * b_bytes) + c * 256, lbo, sbo);
                            mma_bf16(tmem + (uint32_t)(g * Np), da, db, id, (first && c == 0) ? 0u : 1u);
                        }
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&bars[1])));
            } else {
                ok = false;
                atomicExch(err, 1);
                // let the copy in flight land before the shared memory can be reused
                mbar_wait(&bars[0], kc & 1);
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bars[1])) : "memory");
            }
        }
    }
    if (!mbar_wait(&bars[1], (nchunks - 1) & 1)) ok = false;
    if (!ok && (tid & 31) == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;");

    // epilogue: thread tid owns TMEM lane tid (= its line); 8 output columns at a time
    for (int cb = 0; cb < Np; cb += 8) {
        uint32_t r[NACC][8];
#pragma unroll
        for (int g = 0; g < NACC; g++) {
            const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(g * Np + cb);
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(r[g][0]), "=r"(r[g][1]), "=r"(r[g][2]), "=r"(r[g][3]), "=r"(r[g][4]),
                           "=r"(r[g][5]), "=r"(r[g][6]), "=r"(r[g][7])
                         : "r"(ta));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (ok && valid) {
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int i = cb + j;
                if (i < N) {
                    double v;
                    if (line_bad) v = __longlong_as_double(0x7FF8000000000000ll);
                    else {
                        const long long R = combine(__uint_as_float(r[0][j]), __uint_as_float(r[1][j]),
                                                    __uint_as_float(r[2][j]), __uint_as_float(r[3][j]),
                                                    __uint_as_float(r[4][j]));
                        v = ldexp_int(R, EL + sF[i] - 2096);
                    }
                    double* p = job.dst + base + (long long)i * stride;
                    if (job.accumulate) *p += v;
                    else *p = v;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

void fx_geometry(int N, int* Np, int* Kp, int* KC) {
    *Kp = (N + 15) / 16 * 16;
    *Np = *Kp;
    *KC = (*Kp % 32 == 0) ? 32 : 16;
}

size_t fx_smem_bytes(int N) {
    int Np, Kp, KC;
    fx_geometry(N, &Np, &Kp, &KC);
    return (size_t)NDIG * (128u * KC * 2 + (size_t)Np * KC * 2) + (size_t)Np * 4 + 2 * sizeof(uint64_t) + 16;
}

bool fx_supported(int dir, int N) { return N >= 2 && N <= 64 && (dir != 2 || (N % 2) == 0); }

template <int DIR>
static cudaError_t set_attr_fx() {
    return cudaFuncSetAttribute(k_contract_fx<DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)fx_smem_bytes(64));
}

cudaError_t fx_init() {
    cudaError_t e;
    if ((e = set_attr_fx<0>()) != cudaSuccess) return e;
    if ((e = set_attr_fx<1>()) != cudaSuccess) return e;
    return set_attr_fx<2>();
}

cudaError_t launch_contract_fx(int dir, const Dims& d, const DerivJob* jobs, int njobs, const uint8_t* img,
                               long long img_estride, int* err, cudaStream_t s) {
    if (njobs <= 0) return cudaSuccess;
    const int N = dir == 0 ? d.Nr : (dir == 1 ? d.Nt : d.Np);
    if (!fx_supported(dir, N)) return cudaErrorNotSupported;
    int Np, Kp, KC;
    fx_geometry(N, &Np, &Kp, &KC);
    const int need = NACC * Np;
    const int cols = need <= 32 ? 32 : (need <= 64 ? 64 : (need <= 128 ? 128 : (need <= 256 ? 256 : 512)));
    const size_t sm = fx_smem_bytes(N);
    long long nb;
    if (dir == 0) nb = (long long)d.E * ((d.NtNp + 127) / 128);
    else if (dir == 1) nb = ((long long)d.E * d.Nr * d.Np + 127) / 128;
    else nb = (d.P / N + 127) / 128;
    if (nb <= 0) return cudaSuccess;
    if (nb > 0x7FFFFFFFLL) return cudaErrorInvalidValue;
    dim3 grid((unsigned)nb, (unsigned)njobs);
    if (dir == 0) k_contract_fx<0><<<grid, 128, sm, s>>>(d, jobs, img, img_estride, N, Np, Kp, KC, cols, err);
    else if (dir == 1) k_contract_fx<1><<<grid, 128, sm, s>>>(d, jobs, img, 0, N, Np, Kp, KC, cols, err);
    else k_contract_fx<2><<<grid, 128, sm, s>>>(d, jobs, img, 0, N, Np, Kp, KC, cols, err);
    return cudaGetLastError();
}

}  // namespace gk
