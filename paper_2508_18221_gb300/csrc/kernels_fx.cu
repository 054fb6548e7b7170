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
//     a fifth.  The tensor core adds terms of different magnitude with a truncating
//     alignment, so only the fifth accumulator rounds, about 2^-23 of its own size (2^-40
//     below the leading term) per addition (measured: folding from q + l = 5 on instead
//     costs 1e-12 of the bound below);
//   * the epilogue adds the five accumulators as a 64-bit integer and builds the IEEE
//     double with integer instructions (no FP64 arithmetic: GB300 runs FP64 at ~2 fused
//     operations per SM clock, integer and FP32 work at 64-128).
// Error: below 2e-14 of sum_j |D_ij| max_j |u_j| (tested), a few times the worst-case
// bound of an FP64 dot product of these lengths.  A line holding Inf or NaN yields NaN
// outputs; values below 2^-1022 (subnormals) enter as zero.
//
// Work item: 128 lines (tile) of one field (job) x K <= 64, processed in K chunks of
// KC = 16.  The kernel is persistent: two CTAs per SM (one when five accumulators of 64
// columns need all 512 TMEM columns) loop over the work items, each holding its TMEM
// accumulators for its lifetime and staging the next item's FP64 tile while it computes
// the current one.  The operator's seven digit slices for a chunk are
// prepared on the host in the K-major core-matrix layout (8 rows x 16 bytes per core
// matrix) and fetched with one cp.async.bulk; the line digits are formed by the threads
// from the FP64 bits.  Waits are bounded and report through *err.
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

// R * 2^X: one correctly rounded integer-to-double conversion, then the power of two is
// added to the exponent field (ldexp_int below when the result leaves the normal range)
__device__ __forceinline__ double ldexp_int(long long R, int X);
__device__ __forceinline__ double scale_int(long long R, int X) {
    const double v = __ll2double_rn(R);
    const long long bits = __double_as_longlong(v);
    const int be = (int)((bits >> 52) & 0x7FF) + X;
    if (v != 0.0 && be >= 1 && be <= 2046) return __longlong_as_double(bits + ((long long)X << 52));
    return v == 0.0 ? 0.0 : ldexp_int(R, X);
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
// multiple of 2^-8, g4 of 2^-16, g5 of 2^-24 (all exact: |g_s 2^(8 (s-2))| <= 2^22 for
// K <= 64, < 2^24 for K <= 128), gf carries the rounded low-order terms (|gf| < 2^-8).
__device__ __forceinline__ long long combine(float g2, float g3, float g4, float g5, float gf, bool wide) {
    const float MAG = 12582912.f;  // 1.5 * 2^23: float -> nearest integer for |x| <= 2^22
    const int n2 = __float_as_int(g2 + MAG) - 0x4B400000;
    const int n3 = __float_as_int(fmaf(g3, 256.f, MAG)) - 0x4B400000;
    // K > 64: g4, g5 scaled reach 2^23 (exact integers below 2^24): plain conversions
    const int n4 = wide ? __float2int_rn(g4 * 65536.f) : __float_as_int(fmaf(g4, 65536.f, MAG)) - 0x4B400000;
    const int n5 = wide ? __float2int_rn(g5 * 16777216.f) : __float_as_int(fmaf(g5, 16777216.f, MAG)) - 0x4B400000;
    const float fh = fmaf(gf, 16777216.f, MAG);
    const int nfh = __float_as_int(fh) - 0x4B400000;
    const float flo = fmaf(gf, 16777216.f, -(fh - MAG));  // exact remainder in [-1/2, 1/2]
    const int nlo = __float_as_int(fmaf(flo, 65536.f, MAG)) - 0x4B400000;
    const long long a = ((long long)n2 << 24) + ((long long)n3 << 16) + ((long long)n4 << 8) + (long long)(n5 + nfh);
    return (a << 16) + (long long)nlo;
}

}  // namespace

// The tile's FP64 values are staged in shared memory by bulk copies issued from warp 0
// (all bytes of the tile in flight at once), then read twice: for the line exponent and
// for the digits.  Staging layouts, chosen for conflict-free reads by one thread per line:
//   r, theta: [k][128 lines] (one copy per radial row / per theta row and element slab)
//   phi:      [line][rs x 16 bytes] with rs = (N/2) | 1 (odd row stride in 16-byte units)
struct FxTile {
    long long t0;        // first line (global line index, or line within the element for r)
    int e;               // element (r only)
    int nlines;          // valid lines of the tile
};

template <int DIR>
__device__ __forceinline__ int stg_rs(int N) { return DIR == 2 ? ((N / 2) | 1) : 0; }

// number of bulk copies of a tile and the k-th of them (global source, staging offset in
// doubles, bytes)
template <int DIR>
__device__ __forceinline__ int stg_ncopies(const Dims& d, const FxTile& tl, int N) {
    if (DIR == 0) return N;
    if (DIR == 1) {
        const long long e0 = tl.t0 / d.Np, e1 = (tl.t0 + tl.nlines - 1) / d.Np;
        return (int)(e1 - e0 + 1) * N;
    }
    return tl.nlines;
}
template <int DIR>
__device__ __forceinline__ void stg_copy(const Dims& d, const FxTile& tl, int N, int c, long long* src_off,
                                         int* dst_off, int* bytes) {
    if (DIR == 0) {
        *src_off = (long long)tl.e * d.elem + (long long)c * d.NtNp + tl.t0;
        *dst_off = c * 128;
        *bytes = tl.nlines * 8;
    } else if (DIR == 1) {
        const int seg = c / N, k = c - seg * N;
        const long long eil = tl.t0 / d.Np + seg;
        const long long lo = max(tl.t0, eil * d.Np), hi = min(tl.t0 + tl.nlines, (eil + 1) * d.Np);
        *src_off = eil * d.NtNp + (long long)k * d.Np + (lo - eil * d.Np);
        *dst_off = k * 128 + (int)(lo - tl.t0);
        *bytes = (int)(hi - lo) * 8;
    } else {
        *src_off = (tl.t0 + c) * N;
        *dst_off = c * stg_rs<DIR>(N) * 2;
        *bytes = N * 8;
    }
}
template <int DIR>
__device__ __forceinline__ double stg_at(const double* stg, int m, int k, int N) {
    return DIR == 2 ? stg[m * stg_rs<DIR>(N) * 2 + k] : stg[k * 128 + m];
}

// 256 threads: warp w serves TMEM lane quadrant w & 3 (lines 32 (w & 3) .. + 31, one line
// per lane) and half h = w >> 2 of the work of each line: digits of K values 8h .. 8h + 7
// of every 16-wide K chunk, output columns h Np/2 .. (h + 1) Np/2 - 1 in the epilogue.
//
// Shared memory (bytes): [nstg staging buffers | A digits 7 x 128 x 16 x 2 |
//   B digits 7 x Np x 16 x 2 | row exponents Np x 4 | line exponents 2 x 128 x 4 |
//   mbarriers (staging x2, B, MMA) | tmem address]
struct FxParams {
    const DerivJob* jobs;
    const uint8_t* img;
    long long img_estride;
    int N, Np, Kp, tmem_cols, nstg, njobs;
    int Npp;                 // output columns per pass (Np, or 64 when Np = 128)
    long long ntiles;
    uint32_t stg_bytes;
    int* err;
};

template <int DIR>
__device__ __forceinline__ void fx_tile(const Dims& d, long long b, int N, FxTile* tl) {
    if (DIR == 0) {
        const long long tpe = (d.NtNp + 127) / 128;
        tl->e = (int)(b / tpe);
        tl->t0 = (b - (long long)tl->e * tpe) * 128;
        tl->nlines = (int)min(128LL, d.NtNp - tl->t0);
    } else {
        const long long nl = DIR == 1 ? (long long)d.E * d.Nr * d.Np : d.P / N;
        tl->e = 0;
        tl->t0 = b * 128;
        tl->nlines = (int)min(128LL, nl - tl->t0);
    }
}

// warp 0: issue the bulk copies of one tile into a staging buffer (lane 0 first announces
// the byte count on the buffer's barrier)
template <int DIR>
__device__ __forceinline__ void fx_stage(const Dims& d, const FxTile& tl, int N, const double* src, double* buf,
                                         uint64_t* bar, int lane) {
    const int nc = stg_ncopies<DIR>(d, tl, N);
    if (lane == 0) {
        uint32_t total = 0;
        for (int c = 0; c < nc; c++) {
            long long so; int dof, by;
            stg_copy<DIR>(d, tl, N, c, &so, &dof, &by);
            total += (uint32_t)by;
        }
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(total)
                     : "memory");
    }
    __syncwarp();
    for (int c = lane; c < nc; c += 32) {
        long long so; int dof, by;
        stg_copy<DIR>(d, tl, N, c, &so, &dof, &by);
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_u32(buf + dof)),
                     "l"(src + so), "r"((uint32_t)by), "r"(smem_u32(bar))
                     : "memory");
    }
}

template <int DIR>
__global__ void __launch_bounds__(256) k_contract_fx(Dims d, FxParams fp) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, half = warp >> 2;
    const int m = quad * 32 + lane;  // this thread's line within the tile
    const int N = fp.N, Np = fp.Np;
    constexpr int KC = 16, kcores = 2;
    const uint32_t a_bytes = 128u * KC * 2;
    const uint32_t b_bytes = (uint32_t)Np * KC * 2;
    const uint32_t chunk_bytes = NDIG * b_bytes;
    const int nchunks = fp.Kp / KC;
    uint8_t* sA = sm + fp.nstg * fp.stg_bytes;
    uint8_t* sB = sA + NDIG * a_bytes;
    int* sF = reinterpret_cast<int*>(sB + chunk_bytes);
    int* sEL = sF + Np;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sEL + 256);  // [0,1] staging, [2] B, [3] MMA
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 4);
    const long long nitems = fp.ntiles * fp.njobs;

    if (tid == 0) {
        for (int b = 0; b < 4; b++) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[b])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(fp.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    bool ok = true;
    uint32_t n_commit = 0, n_bload = 0;  // completed phases of the MMA and B barriers
    long long it = blockIdx.x;
    if (warp == 0 && it < nitems) {
        FxTile t;
        fx_tile<DIR>(d, it % fp.ntiles, N, &t);
        fx_stage<DIR>(d, t, N, fp.jobs[it / fp.ntiles].src, reinterpret_cast<double*>(sm), &bars[0], lane);
    }
    for (int li = 0; it < nitems; it += gridDim.x, li++) {
        const int buf = li % fp.nstg;
        const double* stg = reinterpret_cast<const double*>(sm + buf * fp.stg_bytes);
        const long long nxt = it + gridDim.x;
        const DerivJob job = fp.jobs[it / fp.ntiles];
        FxTile tl;
        fx_tile<DIR>(d, it % fp.ntiles, N, &tl);
        // with two staging buffers the next item's tile is fetched now (its buffer was last
        // read by the previous item, before that item's final MMA)
        if (fp.nstg == 2 && warp == 0 && nxt < nitems) {
            FxTile t;
            fx_tile<DIR>(d, nxt % fp.ntiles, N, &t);
            fx_stage<DIR>(d, t, N, fp.jobs[nxt / fp.ntiles].src,
                          reinterpret_cast<double*>(sm + (buf ^ 1) * fp.stg_bytes), &bars[buf ^ 1], lane);
        }
        long long base;
        long long stride;
        const uint8_t* op = fp.img;
        if (DIR == 0) {
            base = (long long)tl.e * d.elem + tl.t0 + m;
            stride = d.NtNp;
            op = fp.img + tl.e * fp.img_estride;
        } else {
            const long long t = tl.t0 + m;
            if (DIR == 1) {
                const long long eil = t / d.Np;
                base = eil * d.NtNp + (t - eil * d.Np);
                stride = d.Np;
            } else {
                base = t * N;
                stride = 1;
            }
        }
        const bool valid = m < tl.nlines;
        const int* op_exp = reinterpret_cast<const int*>(op + (size_t)nchunks * chunk_bytes);
        for (int n = tid; n < Np; n += 256) sF[n] = op_exp[n];
        if (!mbar_wait(&bars[buf], (uint32_t)((li / fp.nstg) & 1))) ok = false;

        // the line's largest biased exponent (each half scans half of the line)
        {
            int el = 0;
            if (valid)
                for (int j = half; j < N; j += 2)
                    el = max(el, (int)((__double_as_longlong(stg_at<DIR>(stg, m, j, N)) >> 52) & 0x7FF));
            sEL[half * 128 + m] = el;
        }
        __syncthreads();
        const int EL = max(sEL[m], sEL[128 + m]);
        const bool line_bad = EL == 0x7FF;

        const int Npp = fp.Npp, npass = Np / Npp;
        for (int ch = 0; ch < npass; ch++) {
        for (int kc = 0; kc < nchunks; kc++) {
            // the previous MMAs (previous chunk, pass or item) have finished reading A and B
            if (n_commit > 0 && !mbar_wait(&bars[3], (n_commit - 1) & 1)) ok = false;
            if (tid == 0) {
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bars[2])),
                             "r"(chunk_bytes) : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(sB)),
                    "l"(op + (size_t)kc * chunk_bytes), "r"(chunk_bytes), "r"(smem_u32(&bars[2]))
                    : "memory");
            }
            // this half's 8 K values of the chunk: one 16-byte core-matrix row per digit
            {
                const int k0 = kc * KC + half * 8;
                uint32_t w[NDIG][4];
                if (k0 >= N || !valid) {
#pragma unroll
                    for (int q = 0; q < NDIG; q++) w[q][0] = w[q][1] = w[q][2] = w[q][3] = 0u;
                } else {
#pragma unroll
                    for (int h = 0; h < 4; h++) {
                        const int k = k0 + 2 * h;
                        const double u0 = k < N ? stg_at<DIR>(stg, m, k, N) : 0.0;
                        const double u1 = k + 1 < N ? stg_at<DIR>(stg, m, k + 1, N) : 0.0;
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
                }
                const uint32_t off = (uint32_t)(((m >> 3) * kcores + half) * 128 + (m & 7) * 16);
#pragma unroll
                for (int q = 0; q < NDIG; q++)
                    *reinterpret_cast<uint4*>(sA + q * a_bytes + off) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;");
            // with one staging buffer the next item's tile is fetched once the last chunk of
            // this one is converted
            if (fp.nstg == 1 && ch == npass - 1 && kc == nchunks - 1 && warp == 0 && nxt < nitems) {
                FxTile t;
                fx_tile<DIR>(d, nxt % fp.ntiles, N, &t);
                fx_stage<DIR>(d, t, N, fp.jobs[nxt / fp.ntiles].src, reinterpret_cast<double*>(sm), &bars[0],
                              lane);
            }
            if (tid == 0) {
                if (mbar_wait(&bars[2], n_bload & 1)) {
                    const uint32_t id = instr_desc_bf16(128, Npp);
                    const uint32_t lbo = 128u, sbo = (uint32_t)kcores * 128u;
                    // this pass's operator rows ch Npp .. : whole 8-row core-matrix groups
                    const uint32_t brow = (uint32_t)(ch * Npp / 8) * sbo;
                    // digit pairs (q, l), 0-based, s = q + l <= 6 into accumulator min(s, 4);
                    // within the folded accumulator the smallest terms first
                    for (int sd = NDIG - 1; sd >= 0; sd--) {
                        const int g = sd < NACC - 1 ? sd : NACC - 1;
                        for (int q = 0; q <= sd; q++) {
                            const int l = sd - q;
                            const bool first = kc == 0 && q == 0 && (sd < NACC - 1 || sd == NDIG - 1);
                            const uint64_t da = smem_desc(smem_u32(sA + q * a_bytes), lbo, sbo);
                            const uint64_t db = smem_desc(smem_u32(sB + l * b_bytes) + brow, lbo, sbo);
                            mma_bf16(tmem + (uint32_t)(g * Npp), da, db, id, first ? 0u : 1u);
                        }
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_u32(&bars[3])));
                } else {
                    ok = false;
                    atomicExch(fp.err, 1);
                    // let the copy in flight land before the shared memory is reused
                    mbar_wait(&bars[2], n_bload & 1);
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bars[3])) : "memory");
                }
            }
            n_bload++;
            n_commit++;
        }
        if (!mbar_wait(&bars[3], (n_commit - 1) & 1)) ok = false;
        asm volatile("tcgen05.fence::after_thread_sync;");

        // epilogue: TMEM lane m (this thread's line), this half's output columns of the
        // pass, 8 at a time
        const int c0 = ch * Npp + half * (Npp / 2), c1 = c0 + Npp / 2;
        for (int cb = c0; cb < c1; cb += 8) {
            uint32_t r[NACC][8];
#pragma unroll
            for (int g = 0; g < NACC; g++) {
                const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(g * Npp + cb - ch * Npp);
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(r[g][0]), "=r"(r[g][1]), "=r"(r[g][2]), "=r"(r[g][3]), "=r"(r[g][4]),
                               "=r"(r[g][5]), "=r"(r[g][6]), "=r"(r[g][7])
                             : "r"(ta));
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (ok && valid) {
                double v[8];
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    const long long R = combine(__uint_as_float(r[0][j]), __uint_as_float(r[1][j]),
                                                __uint_as_float(r[2][j]), __uint_as_float(r[3][j]),
                                                __uint_as_float(r[4][j]), fp.Kp > 64);
                    v[j] = scale_int(R, EL + sF[cb + j] - 2096);
                }
                if (line_bad)
#pragma unroll
                    for (int j = 0; j < 8; j++) v[j] = __longlong_as_double(0x7FF8000000000000ll);
                double* p = job.dst + base + (long long)cb * stride;
                if (job.accumulate) {
#pragma unroll
                    for (int j = 0; j < 8; j++)
                        if (cb + j < N) p[(long long)j * stride] += v[j];
                } else {
#pragma unroll
                    for (int j = 0; j < 8; j++)
                        if (cb + j < N) p[(long long)j * stride] = v[j];
                }
            }
        }
        // TMEM (and, after the last pass, sF and sEL) free for the next pass or item
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        }
    }
    if (!ok && lane == 0) atomicExch(fp.err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(fp.tmem_cols));
}

// K padded to 16; output rows padded to K (<= 64) or to 128 (two passes of 64 columns)
void fx_geometry(int N, int* Np, int* Kp, int* KC) {
    *Kp = (N + 15) / 16 * 16;
    *Np = *Kp <= 64 ? *Kp : 128;
    *KC = 16;
}

bool fx_supported(int dir, int N) { return N >= 2 && N <= 128 && (dir != 2 || (N % 2) == 0); }

static uint32_t fx_stg_bytes(int dir, int N) {
    if (dir == 2) return 128u * (uint32_t)((N / 2) | 1) * 16u;
    return 128u * (uint32_t)N * 8u;
}

// everything but the staging buffers
static size_t fx_rest_bytes(int Np) {
    return (size_t)NDIG * (128u * 16 * 2 + (size_t)Np * 16 * 2) + (size_t)Np * 4 + 256 * 4 + 4 * sizeof(uint64_t) + 16;
}

// CTAs per SM (TMEM: 5 Np columns, rounded to a power of two, from 512), staging buffers
// (two when they fit the per-CTA share of the SM's 228 KB, 1 KB reserved per CTA) and the
// dynamic shared memory, at least 1/(ctas + 1) of the SM so that no further CTA co-resides
// (its TMEM allocation would wait for a CTA to finish all of its work)
struct FxCfg {
    int cols, ctas, nstg;
    size_t smem;
};
static FxCfg fx_cfg(int dir, int N) {
    int Np, Kp, KC;
    fx_geometry(N, &Np, &Kp, &KC);
    FxCfg c;
    const int Npp = Np > 64 ? 64 : Np;
    const int need = NACC * Npp;
    c.cols = need <= 32 ? 32 : (need <= 64 ? 64 : (need <= 128 ? 128 : (need <= 256 ? 256 : 512)));
    c.ctas = c.cols <= 256 ? 2 : 1;
    const size_t share = 233472 / c.ctas - 1024;
    const size_t stg = fx_stg_bytes(dir, N), rest = fx_rest_bytes(Np);
    c.nstg = 2 * stg + rest <= share ? 2 : 1;
    const size_t b = c.nstg * stg + rest;
    const size_t floor_ = 233472 / (c.ctas + 1) + 1;
    c.smem = b > floor_ ? b : floor_;
    return c;
}

size_t fx_smem_bytes(int dir, int N) { return fx_cfg(dir, N).smem; }

static size_t fx_smem_max(int dir) {
    size_t mx = 0;
    for (int n = 2; n <= 128; n++) mx = fx_smem_bytes(dir, n) > mx ? fx_smem_bytes(dir, n) : mx;
    return mx;
}

template <int DIR>
static cudaError_t set_attr_fx() {
    return cudaFuncSetAttribute(k_contract_fx<DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)fx_smem_max(DIR));
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
    FxParams fp;
    fp.jobs = jobs;
    fp.img = img;
    fp.img_estride = dir == 0 ? img_estride : 0;
    fp.N = N;
    fp.Np = Np;
    fp.Kp = Kp;
    fp.Npp = Np > 64 ? 64 : Np;
    const FxCfg cfg = fx_cfg(dir, N);
    fp.tmem_cols = cfg.cols;
    fp.nstg = cfg.nstg;
    fp.njobs = njobs;
    fp.stg_bytes = fx_stg_bytes(dir, N);
    fp.err = err;
    if (dir == 0) fp.ntiles = (long long)d.E * ((d.NtNp + 127) / 128);
    else if (dir == 1) fp.ntiles = ((long long)d.E * d.Nr * d.Np + 127) / 128;
    else fp.ntiles = (d.P / N + 127) / 128;
    if (fp.ntiles <= 0) return cudaSuccess;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long nitems = fp.ntiles * njobs;
    const long long grid = nitems < (long long)cfg.ctas * nsm ? nitems : (long long)cfg.ctas * nsm;
    const size_t sm = cfg.smem;
    if (dir == 0) k_contract_fx<0><<<(unsigned)grid, 256, sm, s>>>(d, fp);
    else if (dir == 1) k_contract_fx<1><<<(unsigned)grid, 256, sm, s>>>(d, fp);
    else k_contract_fx<2><<<(unsigned)grid, 256, sm, s>>>(d, fp);
    return cudaGetLastError();
}

}  // namespace gk
