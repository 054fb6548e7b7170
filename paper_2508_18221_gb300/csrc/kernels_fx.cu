// FP64-accurate spectral contractions on the 16-bit tensor cores (tcgen05, sm_103a).
//
// out[line][i] = sum_j D[i][j] u[line][j] in double precision, computed with the
// error-free splitting of Ozaki, Ogita, Oishi & Rump (Numer. Algorithms 59, 2012):
//   * every line of u gets one common exponent (its largest), every row of D its own;
//     relative to it each value is a signed 54-bit fixed-point integer, written as seven
//     balanced base-256 digits d_1..d_7 in [-128, 127] (most significant first);
//   * a digit fits an FP16 exactly and a product of two digits (|.| <= 2^14) fits an FP32
//     exactly, so the tensor core forms sum_j c_l(i,j) d_q(j) without rounding as long as
//     the running sum stays below 2^24 (true for K <= 128 and the sums below);
//   * the 28 digit pairs with q + l <= 8 are kept, each digit-order sum s = q + l = 2..8 in
//     a TMEM accumulator of its own, so every accumulator is exact (|sum| < 2^24 units of
//     its order for K <= 128: at most 7 pairs of products below 2^14);
//   * the operator's seven slices of one K chunk form one tall matrix (slice after slice),
//     so the products of line slice q with operator slices 1 .. 8 - q are one MMA whose
//     N = (8 - q) Npp output columns start at accumulator q + 1: seven MMAs per chunk (a
//     few more where N would pass 256) instead of one per pair;
//   * the epilogue adds the seven accumulators as a 64-bit integer (the s = 8 term rounded
//     to the s = 7 unit) and builds the IEEE double with one integer-to-double conversion
//     and an exponent add (GB300 runs FP64 at ~2 fused operations per SM clock, integer
//     and FP32 work at 64-128).
// Error: about 1e-15 of sum_j |D_ij| max_j |u_j| (the dropped pairs q + l > 8 and the final
// roundings), below the worst-case bound of an FP64 dot product of these lengths.  A line
// holding Inf or NaN yields NaN outputs; values below 2^-1022 (subnormals) enter as zero.
//
// Work item: 128 lines (tile) of one field (job) x K <= 128, one pass of at most 64 output
// columns, processed in K chunks of 16.  The kernel is persistent and warp-specialised
// (roles below k_contract_fx): two CTAs per SM up to 32 nodes, one above, each holding
// its TMEM accumulators for its lifetime.  The operator's seven digit slices are prepared
// on the host in the K-major core-matrix layout (8 rows x 16 bytes per core matrix) and
// fetched by cp.async.bulk; the line digits are formed by the converter warps from the
// FP64 bits.  Waits are bounded in time and report through *err.
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>

#include "grmhd_internal.h"

namespace gk {

namespace {

constexpr int NDIG = 7;                                      // base-256 digits per operand
constexpr int NACC = 7;                                      // TMEM accumulators: s = 2..8
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

// D = F32, A = B = F16, both K-major; N >> 3 at bit 17, M >> 4 at bit 24
__device__ __forceinline__ uint32_t instr_desc_f16(int m, int n) {
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}


__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t id, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                 "l"(da), "l"(db), "r"(id), "r"(acc));
}

// Digit word of one value: Z = X + bias with X = round(2 m 2^(e - EL)) the value as a
// signed fixed-point integer relative to the line exponent EL (|X| <= 2^54; the value is
// X 2^(EL - 1076)); byte b of Z minus 128 is the balanced digit of weight 256^b.  Branch-
// free (the values of a thread overlap): round(2 m / 2^sh) = ((4 m >> sh) + 1) >> 1 for
// sh = EL - e in 0 .. 63 (4 m < 2^56, so every sh >= 56 gives 0), zero for e = 0.
__device__ __forceinline__ unsigned long long digit_word(double u, int EL) {
    const long long bits = __double_as_longlong(u);
    const int e = (int)((bits >> 52) & 0x7FF);
    const unsigned long long m4 = (((unsigned long long)bits & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 2;
    const int sh = min(EL - e, 63);
    const unsigned long long mag = e != 0 ? ((m4 >> sh) + 1) >> 1 : 0ull;
    const long long x = bits < 0 ? -(long long)mag : (long long)mag;
    return (unsigned long long)(x + (long long)DIG_BIAS);
}

// Digit words of a value pair (u0, u1) for the A operand: FP16x2 words holding digit q of
// u0 (low half) and of u1 (high half).  A biased digit byte b is placed under the byte
// 0x64, giving the FP16 number 1024 + b, and one packed FP16 add of -1152 leaves b - 128
// exactly.  Per value, four byte permutes spread its digit bytes over halves whose high
// byte is 0x64 (e: bytes 0 and 2, o: bytes 1 and 3 of each 32-bit word of Z); per digit,
// one permute pairs the two values and one packed add removes the bias.
struct DigitHalves {
    uint32_t el, ol, eh, oh;
};
__device__ __forceinline__ DigitHalves digit_halves(unsigned long long z) {
    const uint32_t l = (uint32_t)z, h = (uint32_t)(z >> 32), C = 0x64646464u;
    return {__byte_perm(l, C, 0x4240), __byte_perm(l, C, 0x4341), __byte_perm(h, C, 0x4240),
            __byte_perm(h, C, 0x4441)};
}
__device__ __forceinline__ uint32_t unbias(uint32_t w) {
    uint32_t r;
    asm("add.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(w), "r"(0xE480E480u));  // -1152 in both halves
    return r;
}

// R * 2^X: one correctly rounded integer-to-double conversion, then the power of two is
// added to the exponent field; *ok false when the result leaves the normal range or R = 0
// (the caller then takes ldexp_int below).  Branch-free, so that the eight outputs of a
// column block overlap their conversions.
__device__ __forceinline__ double ldexp_int(long long R, int X);
__device__ __forceinline__ double scale_int_fast(long long R, int X, bool* ok) {
    const double v = __ll2double_rn(R);
    const int lo = __double2loint(v), hi = __double2hiint(v);
    const int e = (hi >> 20) & 0x7FF;
    *ok = e != 0 && (unsigned)(e + X - 1) < 2046u;
    return __hiloint2double(hi + (X << 20), lo);
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

// T = sum_s n_s 2^(-8 (s - 2)) as the integer R = round(T 2^40), n_s = acc[s - 2] the exact
// integer sum of the digit products of order s (digits are plain integers in both
// operands), |n_s| <= (s - 1) K 2^14: below 2^24 for K <= 128 and below 2^22 for K <= 32.
// Each n_s is made non-negative by an offset, t_s = n_s + o_s: below 2^22 t_s is read off
// the bits of n_s + 1.5 * 2^23 (the low 23 bits hold n_s + 2^22; exact, as n_s is an
// integer), above it comes from a float-to-integer conversion (exact too).
// The t_s are summed at their byte offsets with 32 x 32 -> 64-bit multiply-adds (an
// unsigned sum below 2^63), the s = 8 term rounded to the unit of s = 7 (half up), and the
// offsets' total is subtracted once.
template <bool WIDE>
__device__ __forceinline__ long long combine7(const uint32_t* acc) {
    const float MAG = 12582912.f;  // 1.5 * 2^23
    uint32_t t[NACC];
    unsigned long long off;
    if (!WIDE) {
#pragma unroll
        for (int s = 0; s < NACC; s++) t[s] = (uint32_t)__float_as_int(__uint_as_float(acc[s]) + MAG) & 0x7FFFFFu;
        // o_s = 2^22 for every s
        off = (1ull << 62) + (1ull << 54) + (1ull << 46) + (1ull << 38) + (1ull << 30) + (1ull << 22) + (1ull << 14);
    } else {
        // |n_s| <= (s - 1) K 2^14 <= (s - 1) 2^21: o_2 = 2^21, the others o_s = 2^24
#pragma unroll
        for (int s = 0; s < NACC; s++)
            t[s] = (uint32_t)(__float2int_rn(__uint_as_float(acc[s])) + (s == 0 ? (1 << 21) : (1 << 24)));
        off = (1ull << 61) + (1ull << 56) + (1ull << 48) + (1ull << 40) + (1ull << 32) + (1ull << 24) + (1ull << 16);
    }
    // t_2 2^40 + t_3 2^32 + t_4 2^24 + t_5 2^16 + t_6 2^8 + t_7 + round(t_8 / 256)
    unsigned long long a = (unsigned long long)t[2] * (1ull << 24) + t[5];
    a += (unsigned long long)t[3] * (1ull << 16);
    a += (unsigned long long)t[4] * (1ull << 8);
    a += (unsigned long long)((t[0] << 8) + t[1]) << 32;
    a += (t[6] + 128u) >> 8;
    return (long long)(a - off);
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
        const long long eil = (long long)((uint32_t)tl.t0 / (uint32_t)d.Np) + seg;
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

struct FxParams {
    const DerivJob* jobs;
    const uint8_t* img;
    long long img_estride;
    int N, Np, Kp, tmem_cols, nstg, njobs;
    int Npp;                 // output columns per pass (Np, or 64 when Np = 128)
    int npass;               // Np / Npp
    int b_all;               // 1: the operator digits of all K chunks stay in shared memory
    long long ntiles;        // 128-line tiles of one field
    uint32_t per_job;        // items of one field: ntiles x npass
    uint32_t tpe;            // radial: 128-line tiles per element
    uint32_t nlf;            // lines of one field (theta, phi)
    uint32_t stg_bytes;
    int* err;
    int stall;               // test of the wait limits: the staging warp issues no copies
    int tsets;               // TMEM accumulator sets: 1, or 2 (item k in set k % 2: the MMAs of
                             // item k + 1 run while the epilogue drains item k; needs b_all)
};

// tile b of a field (32-bit arithmetic: a field holds fewer than 2^31 points, since its 32
// or 33 fields fit the device memory)
template <int DIR>
__device__ __forceinline__ void fx_tile(const FxParams& fp, const Dims& d, uint32_t b, FxTile* tl) {
    if (DIR == 0) {
        const uint32_t e = b / fp.tpe, t0 = (b - e * fp.tpe) * 128u;
        tl->e = (int)e;
        tl->t0 = t0;
        tl->nlines = (int)min(128u, (uint32_t)d.NtNp - t0);
    } else {
        tl->e = 0;
        tl->t0 = b * 128u;
        tl->nlines = (int)min(128u, fp.nlf - b * 128u);
    }
}

// warp 0: issue the bulk copies of one tile into a staging buffer (lane 0 first announces
// the byte count on the buffer's barrier)
template <int DIR>
__device__ __forceinline__ void fx_stage(const Dims& d, const FxTile& tl, int N, const double* src, double* buf,
                                         uint64_t* bar, int lane) {
    const int nc = stg_ncopies<DIR>(d, tl, N);
    if (lane == 0) {
        // the copies cover the tile's lines x N values exactly once
        const uint32_t total = (uint32_t)tl.nlines * (uint32_t)N * 8u;
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


// Warp roles (320 threads):
//   warps 0-3  convert: thread m = line m of the item's tile; line exponent, operator row
//              exponents, then the seven digit slices of each 16-wide K chunk into a
//              two-stage ring of A buffers;
//   warps 4-7  epilogue: thread m reads TMEM lane m (warp w serves lane quadrant w & 3),
//              combines the seven accumulators and stores the FP64 results, 8 columns
//              at a time; TMEM goes back to the MMA warp once the last block is in
//              registers, before its arithmetic (the epilogue's latency, not its
//              instruction count, sets the rate at which items pass through TMEM);
//   warp 8     stages the FP64 tiles in shared memory (bulk copies);
//   warp 9     one thread loads the operator digits and issues the MMAs (per K chunk one
//              per line slice q, over the stacked operator slices 1 .. 8 - q).
// A work item is (field, 128-line tile, column pass); the CTA walks items blockIdx.x,
// blockIdx.x + gridDim.x, ...  Every role follows the same item sequence; they hand over
// through mbarriers (full / empty pairs), so conversion of one item overlaps the MMAs
// and the epilogue of the previous one.  Every wait is bounded in time (globaltimer);
// after a timeout the CTA raises an abort flag, every role leaves its loop, and *err is
// set.
//
// Shared memory (bytes): [staging x nstg | A ring 2 x (7 x 128 x 16 x 2) |
//   B digits of all chunks (nchunks x 7 x Np x 16 x 2) | sEL 2 x 128 x 4 | sF 2 x 128 x 4 |
//   barriers | tmem address | abort flag]
// WC converter warps and WE epilogue warps (multiples of 4), a staging warp and an MMA warp:
// (4, 4) at two CTAs per SM, (8, 8) at one.  (Eight epilogue warps beside four converters at
// two CTAs per SM, 72 registers a thread, spill and were measured slower.)
__host__ __device__ constexpr int fx_threads(int WC, int WE) { return (WC + WE + 2) * 32; }
constexpr int NA_RING = 2;

// exponents and their barriers alternate between two sets by item parity, so that the
// converters write item k's line exponents while the epilogue still reads item k - 1's
struct FxBars {
    uint64_t stg_full[2], stg_empty[2], a_full[NA_RING], a_empty[NA_RING];
    uint64_t acc_full[2], acc_empty[2], el_ready[2], b_full;
};

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait for the phase with the given parity, at most ~0.5 s; false on timeout or abort.
// The suspend-time hint parks the warp in hardware until the phase completes (up to
// 100 us per try), so waiting roles do not take issue slots from working ones.
__device__ __forceinline__ bool bwait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    const uint64_t t0 = gtimer();
    for (;;) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
                     "selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(smem_u32(bar)), "r"(parity), "r"(100000u) : "memory");
        if (done) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > 500000000ull) {
            *abort_flag = 1;
            return false;
        }
    }
}

// wait for a phase regardless of the abort flag, at most `ns` nanoseconds (the wind-down
// after an abort: work issued before it must finish before TMEM is freed)
__device__ __forceinline__ bool bwait_for(uint64_t* bar, uint32_t parity, uint64_t ns) {
    const uint64_t t0 = gtimer();
    for (;;) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
                     "selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(smem_u32(bar)), "r"(parity), "r"(10000u) : "memory");
        if (done) return true;
        if (gtimer() - t0 > ns) return false;
    }
}

__device__ __forceinline__ void barrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// warp-wide bounded wait: every lane polls; the warp goes on only if every lane saw the phase
__device__ __forceinline__ bool wwait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    return __all_sync(0xffffffffu, bwait(bar, parity, abort_flag) ? 1 : 0) != 0;
}

// one lane of the (converged) warp
__device__ __forceinline__ bool elect_one() {
    uint32_t p;
    asm volatile("{\n.reg .pred e;\nelect.sync _|e, 0xffffffff;\nselp.u32 %0, 1, 0, e;\n}\n" : "=r"(p));
    return p != 0;
}

// work item it -> field (job), tile and column pass (npass is 1 or 2); items < 2^31
template <int DIR>
__device__ __forceinline__ void fx_item(const FxParams& fp, const Dims& d, long long it, FxTile* tl, int* pass,
                                        int* job) {
    const uint32_t u = (uint32_t)it, j = u / fp.per_job, r = u - j * fp.per_job;
    *job = (int)j;
    *pass = fp.npass == 2 ? (int)(r & 1u) : 0;
    fx_tile<DIR>(fp, d, fp.npass == 2 ? r >> 1 : r, tl);
}

template <int DIR, int WC, int WE>
__global__ void __launch_bounds__(fx_threads(WC, WE), WC == 4 ? 2 : 1) k_contract_fx(Dims d, FxParams fp) {
    constexpr int NA = NACC;
    extern __shared__ __align__(1024) uint8_t sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = fp.N, Np = fp.Np, Npp = fp.Npp;
    constexpr int KC = 16, kcores = 2;
    const uint32_t a_bytes = 128u * KC * 2;            // one digit slice of one chunk
    const uint32_t a_stage = NDIG * a_bytes;
    const uint32_t b_bytes = (uint32_t)Np * KC * 2;        // one slice of one chunk, all passes
    const uint32_t bs_bytes = (uint32_t)Npp * KC * 2;      // one slice of one chunk and pass
    const uint32_t chunk_bytes = NDIG * b_bytes;
    const int nchunks = fp.Kp / KC;
    const uint32_t op_bytes = (uint32_t)nchunks * chunk_bytes;
    const uint32_t sb_bytes = fp.b_all ? op_bytes : chunk_bytes;
    uint8_t* sA = sm + fp.nstg * fp.stg_bytes;
    uint8_t* sB = sA + NA_RING * a_stage;
    int* sEL = reinterpret_cast<int*>(sB + sb_bytes);   // [2][128]
    int* sF = sEL + 256;                                // [2][128]
    FxBars* bars = reinterpret_cast<FxBars*>(sF + 256);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const long long nitems = fp.ntiles * fp.npass * fp.njobs;

    if (tid == 0) {
        for (int b = 0; b < 2; b++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars->stg_full[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars->stg_empty[b])), "r"(WC));
        }
        for (int a = 0; a < NA_RING; a++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(&bars->a_full[a])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars->a_empty[a])));
        }
        for (int t = 0; t < 2; t++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars->acc_full[t])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars->acc_empty[t])), "r"(WE));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(&bars->el_ready[t])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars->b_full)));
        asm volatile("fence.mbarrier_init.release.cluster;");
        *abort_flag = 0;
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

    if (warp == WC + WE) {
        // ---------------------------------------------------------------- staging
        int k = 0;
        int last_k[2] = {-1, -1};          // last item staged into each buffer
        for (long long it = blockIdx.x; it < nitems; it += gridDim.x, k++) {
            const int b = k % fp.nstg;
            if (k >= fp.nstg) {
                bool ok = true;
                if (lane == 0) ok = bwait(&bars->stg_empty[b], (uint32_t)((k / fp.nstg - 1) & 1), abort_flag);
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                if (!ok) break;
            }
            FxTile tl;
            int pass, job;
            fx_item<DIR>(fp, d, it, &tl, &pass, &job);
            if (!fp.stall) {
                fx_stage<DIR>(d, tl, N, fp.jobs[job].src, reinterpret_cast<double*>(sm + b * fp.stg_bytes),
                              &bars->stg_full[b], lane);
                last_k[b] = k;
            }
        }
        // after an abort, the copies already issued land before the CTA frees its memory
        if (*abort_flag && lane == 0)
            for (int b = 0; b < fp.nstg; b++)
                if (last_k[b] >= 0) bwait_for(&bars->stg_full[b], (uint32_t)((last_k[b] / fp.nstg) & 1), 1000000ull);
    } else if (warp == WC + WE + 1) {
        // ---------------------------------------------------------------- MMA issue
        // The whole warp walks the loop with warp-uniform values (descriptors, columns,
        // counters); one elected lane issues the copies, MMAs and commits.  (Issued from
        // a single-lane branch, each MMA cost ~150 cycles of issue.)
        const bool leader = elect_one();
        const int gmax = 256 / Npp;  // operator slices per MMA (N <= 256)
        const uint32_t lbo = 128u, sbo = (uint32_t)kcores * 128u;
        int k = 0, cur_e = -1;
        uint32_t n_b = 0;
        int last_cg = -1, last_item = -1;   // last chunk / item whose MMAs were committed
        for (long long it = blockIdx.x; it < nitems; it += gridDim.x, k++) {
            FxTile tl;
            int pass, job;
            fx_item<DIR>(fp, d, it, &tl, &pass, &job);
            // the epilogue has drained the accumulator set this item writes (item k - tsets)
            const int ts = fp.tsets;
            if (k >= ts && !wwait(&bars->acc_empty[(k - ts) & 1], (uint32_t)(((k - ts) >> 1) & 1), abort_flag))
                break;
            const uint8_t* op = fp.img + (DIR == 0 ? tl.e * fp.img_estride : 0);
            // with two sets the previous item's MMAs may still read the operator: they
            // finish (its commit) before a new element's operator overwrites it
            if (ts > 1 && k > 0 && fp.b_all && cur_e != tl.e &&
                !wwait(&bars->acc_full[(k - 1) % ts], (uint32_t)(((k - 1) / ts) & 1), abort_flag))
                break;
            if (fp.b_all && cur_e != tl.e) {  // radial: per-element operator; theta, phi: once
                if (leader) {
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                                     smem_u32(&bars->b_full)),
                                 "r"(op_bytes) : "memory");
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            smem_u32(sB)),
                        "l"(op), "r"(op_bytes), "r"(smem_u32(&bars->b_full))
                        : "memory");
                }
                __syncwarp();
                n_b++;
                cur_e = tl.e;
            }
            if (fp.b_all && !wwait(&bars->b_full, (n_b - 1) & 1, abort_flag)) break;
            const uint32_t bpass = (uint32_t)pass * NDIG * bs_bytes;  // this pass's slices
            const uint32_t set_col = (uint32_t)((k % ts) * NA * Npp);
            bool stop = false;
            for (int kc = 0; kc < nchunks; kc++) {
                const int cg = k * nchunks + kc, a = cg % NA_RING;
                if (!fp.b_all) {
                    // one chunk of the operator at a time: the previous chunk's MMAs (the
                    // previous item's are done: acc_empty) have finished reading it
                    if (kc > 0) {
                        const int cp = cg - 1;
                        if (!wwait(&bars->a_empty[cp % NA_RING], (uint32_t)((cp / NA_RING) & 1), abort_flag)) {
                            stop = true;
                            break;
                        }
                    }
                    if (leader) {
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                                         smem_u32(&bars->b_full)),
                                     "r"(chunk_bytes) : "memory");
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                smem_u32(sB)),
                            "l"(op + (size_t)kc * chunk_bytes), "r"(chunk_bytes), "r"(smem_u32(&bars->b_full))
                            : "memory");
                    }
                    __syncwarp();
                    n_b++;
                    if (!wwait(&bars->b_full, (n_b - 1) & 1, abort_flag)) { stop = true; break; }
                }
                if (!wwait(&bars->a_full[a], (uint32_t)((cg / NA_RING) & 1), abort_flag)) { stop = true; break; }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t a0 = smem_u32(sA + a * a_stage);
                const uint32_t b0 = smem_u32(sB + (fp.b_all ? kc * chunk_bytes : 0)) + bpass;
                // line slice q times operator slices l0 .. l0 + c - 1 (consecutive rows of the
                // chunk's tall operator matrix) into accumulators q + l0 .. q + l0 + c - 1;
                // q = 0 of the first chunk writes every accumulator first
                if (leader) {
                    for (int q = 0; q < NDIG; q++)
                        for (int l0 = 0; l0 < NDIG - q; l0 += gmax) {
                            const int c = min(gmax, NDIG - q - l0);
                            mma_f16(tmem + set_col + (uint32_t)((q + l0) * Npp), smem_desc(a0 + q * a_bytes, lbo, sbo),
                                     smem_desc(b0 + l0 * bs_bytes, lbo, sbo), instr_desc_f16(128, c * Npp),
                                     (kc == 0 && q == 0) ? 0u : 1u);
                        }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_u32(&bars->a_empty[a])));
                }
                __syncwarp();
                last_cg = cg;
            }
            if (stop) break;
            if (leader)
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&bars->acc_full[k % ts])));
            __syncwarp();
            last_item = k;
        }
        // after an abort, the MMAs already committed finish writing TMEM, and an operator
        // copy already issued lands, before TMEM and shared memory are given up
        if (*abort_flag && leader) {
            if (last_cg >= 0)
                bwait_for(&bars->a_empty[last_cg % NA_RING], (uint32_t)((last_cg / NA_RING) & 1), 1000000ull);
            if (last_item >= 0)
                bwait_for(&bars->acc_full[last_item % fp.tsets], (uint32_t)((last_item / fp.tsets) & 1), 1000000ull);
            if (n_b > 0) bwait_for(&bars->b_full, (n_b - 1) & 1, 1000000ull);
        }
        __syncwarp();
    } else if (warp < WC) {
        // ---------------------------------------------------------------- conversion
        // thread m = line m; with W = 8 two groups of 4 warps share the K chunks by A ring
        // slot (group g writes the chunks that land in slot g); group 0 publishes exponents
        const int m = tid & 127, grp = tid >> 7;
        int k = 0;
        for (long long it = blockIdx.x; it < nitems; it += gridDim.x, k++) {
            FxTile tl;
            int pass, job;
            fx_item<DIR>(fp, d, it, &tl, &pass, &job);
            const int b = k % fp.nstg;
            const double* stg = reinterpret_cast<const double*>(sm + b * fp.stg_bytes);
            const bool valid = m < tl.nlines;
            if (!bwait(&bars->stg_full[b], (uint32_t)((k / fp.nstg) & 1), abort_flag)) break;
            int EL = 0;
            if (valid)
                for (int j = 0; j < N; j++)
                    EL = max(EL, (int)((__double_as_longlong(stg_at<DIR>(stg, m, j, N)) >> 52) & 0x7FF));
            if (grp == 0) {
                // the epilogue of item k - 2 has read this set of sEL and sF
                const int t = k & 1;
                if (k > 1 && !bwait(&bars->acc_empty[t], (uint32_t)(((k - 2) >> 1) & 1), abort_flag)) break;
                sEL[t * 128 + m] = EL;
                if (m < Np) {
                    const uint8_t* op = fp.img + (DIR == 0 ? tl.e * fp.img_estride : 0);
                    sF[t * 128 + m] = reinterpret_cast<const int*>(op + (size_t)op_bytes)[m];
                }
                __syncwarp();
                if (lane == 0) barrive(&bars->el_ready[t]);
            }
            bool stop = false;
            for (int kc = 0; kc < nchunks; kc++) {
                const int cg = k * nchunks + kc, a = cg % NA_RING;
                if (WC == 8 && a != grp) continue;
                if (cg >= NA_RING && !bwait(&bars->a_empty[a], (uint32_t)((cg / NA_RING - 1) & 1), abort_flag)) {
                    stop = true;
                    break;
                }
                uint8_t* dstA = sA + a * a_stage;
#pragma unroll
                for (int g8 = 0; g8 < kcores; g8++) {
                    const int k0 = kc * KC + g8 * 8;
                    uint32_t w[NDIG][4];
                    if (k0 >= N || !valid) {
#pragma unroll
                        for (int q = 0; q < NDIG; q++) w[q][0] = w[q][1] = w[q][2] = w[q][3] = 0u;
                    } else {
#pragma unroll
                        for (int h = 0; h < 4; h++) {
                            const int kk = k0 + 2 * h;
                            const double u0 = kk < N ? stg_at<DIR>(stg, m, kk, N) : 0.0;
                            const double u1 = kk + 1 < N ? stg_at<DIR>(stg, m, kk + 1, N) : 0.0;
                            const DigitHalves a0 = digit_halves(digit_word(u0, EL));
                            const DigitHalves a1 = digit_halves(digit_word(u1, EL));
                            // digit q = 1 .. 7 sits in byte 7 - q of Z
                            w[0][h] = unbias(__byte_perm(a0.eh, a1.eh, 0x7632));   // byte 6
                            w[1][h] = unbias(__byte_perm(a0.oh, a1.oh, 0x5410));   // byte 5
                            w[2][h] = unbias(__byte_perm(a0.eh, a1.eh, 0x5410));   // byte 4
                            w[3][h] = unbias(__byte_perm(a0.ol, a1.ol, 0x7632));   // byte 3
                            w[4][h] = unbias(__byte_perm(a0.el, a1.el, 0x7632));   // byte 2
                            w[5][h] = unbias(__byte_perm(a0.ol, a1.ol, 0x5410));   // byte 1
                            w[6][h] = unbias(__byte_perm(a0.el, a1.el, 0x5410));   // byte 0
                        }
                    }
                    const uint32_t off = (uint32_t)(((m >> 3) * kcores + g8) * 128 + (m & 7) * 16);
#pragma unroll
                    for (int q = 0; q < NDIG; q++)
                        *reinterpret_cast<uint4*>(dstA + q * a_bytes + off) =
                            make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) barrive(&bars->a_full[a]);
            }
            if (stop) break;
            // this item's staging buffer is no longer read
            __syncwarp();
            if (lane == 0) barrive(&bars->stg_empty[b]);
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        // warp w reads TMEM lanes 32 (w & 3) ..; with W = 8 the two warps of a lane quadrant
        // take the first and the second half of the column blocks
        const int quad = warp & 3, m = quad * 32 + lane, half = (warp - WC) >> 2;
        const bool wide = fp.Kp > 32;   // scaled accumulators reach 2^22
        int k = 0;
        for (long long it = blockIdx.x; it < nitems; it += gridDim.x, k++) {
            FxTile tl;
            int pass, job;
            fx_item<DIR>(fp, d, it, &tl, &pass, &job);
            const DerivJob jb = fp.jobs[job];  // loaded before the waits
            const int t = k & 1;
            if (!bwait(&bars->el_ready[t], (uint32_t)((k >> 1) & 1), abort_flag)) break;
            if (!bwait(&bars->acc_full[k % fp.tsets], (uint32_t)((k / fp.tsets) & 1), abort_flag)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const bool valid = m < tl.nlines;
            long long base, stride;
            if (DIR == 0) {
                base = (long long)tl.e * d.elem + tl.t0 + m;
                stride = d.NtNp;
            } else {
                const long long t = tl.t0 + m;
                if (DIR == 1) {
                    const uint32_t eil = (uint32_t)t / (uint32_t)d.Np;
                    base = (long long)eil * d.NtNp + (t - (long long)eil * d.Np);
                    stride = d.Np;
                } else {
                    base = t * N;
                    stride = 1;
                }
            }
            const int EL = sEL[t * 128 + m];
            const bool line_bad = EL == 0x7FF;
            // column blocks holding output rows of this pass (the padding blocks beyond N are
            // computed by the MMAs but not read)
            const int ncol = min(Npp, N - pass * Npp);
            const int nblk = (ncol + 7) >> 3, nh = WE == 8 ? (nblk + 1) >> 1 : nblk;
            const int cb_beg = half == 0 ? 0 : nh * 8, cb_end = half == 0 ? nh * 8 : nblk * 8;
            const uint32_t set_col = (uint32_t)((k % fp.tsets) * NA * Npp);
            if (cb_beg >= cb_end) {       // no block for this warp: release at once
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0) barrive(&bars->acc_empty[t]);
            }
            for (int cb = cb_beg; cb < cb_end; cb += 8) {
                uint32_t r[NA][8];
#pragma unroll
                for (int g = 0; g < NA; g++) {
                    const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + set_col + (uint32_t)(g * Npp + cb);
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                 : "=r"(r[g][0]), "=r"(r[g][1]), "=r"(r[g][2]), "=r"(r[g][3]), "=r"(r[g][4]),
                                   "=r"(r[g][5]), "=r"(r[g][6]), "=r"(r[g][7])
                                 : "r"(ta));
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                const int c0 = pass * Npp + cb;  // output column of r[.][0]
                int X[8];
#pragma unroll
                for (int j = 0; j < 8; j++) X[j] = EL + sF[t * 128 + c0 + j] - 2096;
                if (cb + 8 >= cb_end) {
                    // every accumulator column has been read, and the row exponents too:
                    // hand TMEM (and this set of sEL, sF) back before the last block's
                    // arithmetic, so that the next item's MMAs start under it
                    asm volatile("tcgen05.fence::before_thread_sync;");
                    __syncwarp();
                    if (lane == 0) barrive(&bars->acc_empty[t]);
                }
                if (valid) {
                    // phases over the eight outputs (combine, convert, fix-ups), so that their
                    // dependency chains overlap
                    long long R[8];
                    if (wide) {
#pragma unroll
                        for (int j = 0; j < 8; j++) {
                            uint32_t acc[NA];
#pragma unroll
                            for (int g = 0; g < NA; g++) acc[g] = r[g][j];
                            R[j] = combine7<true>(acc);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 8; j++) {
                            uint32_t acc[NA];
#pragma unroll
                            for (int g = 0; g < NA; g++) acc[g] = r[g][j];
                            R[j] = combine7<false>(acc);
                        }
                    }
                    double v[8];
                    bool ok[8], all_ok = true;
#pragma unroll
                    for (int j = 0; j < 8; j++) {
                        v[j] = scale_int_fast(R[j], X[j], &ok[j]);
                        all_ok = all_ok && ok[j];
                    }
                    if (!all_ok)
#pragma unroll
                        for (int j = 0; j < 8; j++)
                            if (!ok[j]) v[j] = R[j] == 0 ? 0.0 : ldexp_int(R[j], X[j]);
                    if (line_bad)
#pragma unroll
                        for (int j = 0; j < 8; j++) v[j] = __longlong_as_double(0x7FF8000000000000ll);
                    double* pd = jb.dst + base + (long long)c0 * stride;
                    if (DIR == 2 && c0 + 8 <= N && (reinterpret_cast<uintptr_t>(pd) & 15) == 0) {
                        // phi: the block's outputs are contiguous in the line: 16-byte stores
                        double2* p2 = reinterpret_cast<double2*>(pd);
                        if (jb.accumulate) {
#pragma unroll
                            for (int h = 0; h < 4; h++) {
                                double2 o = p2[h];
                                o.x += v[2 * h];
                                o.y += v[2 * h + 1];
                                p2[h] = o;
                            }
                        } else {
#pragma unroll
                            for (int h = 0; h < 4; h++) p2[h] = make_double2(v[2 * h], v[2 * h + 1]);
                        }
                    } else if (jb.accumulate) {
#pragma unroll
                        for (int j = 0; j < 8; j++)
                            if (c0 + j < N) pd[(long long)j * stride] += v[j];
                    } else {
#pragma unroll
                        for (int j = 0; j < 8; j++)
                            if (c0 + j < N) pd[(long long)j * stride] = v[j];
                    }
                }
            }
        }
    }

    // wind down: every role has left its loop; let bulk copies in flight land, then free TMEM
    __syncthreads();
    if (tid == 0 && *abort_flag) atomicExch(fp.err, 1);
    if (*abort_flag) {
        // the staging and MMA roles waited above for their own copies and MMAs; a further
        // 0.2 ms covers any copy whose barrier phase was already past when they looked
        const uint64_t t0 = gtimer();
        while (gtimer() - t0 < 200000ull) {
        }
    }
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

// everything but the staging buffers: the A ring, B digits (all K chunks when b_all, else
// one chunk), exponents, barriers, TMEM address, abort flag
static size_t fx_rest_bytes(int N, int b_all) {
    int Np, Kp, KC;
    fx_geometry(N, &Np, &Kp, &KC);
    return (size_t)NA_RING * NDIG * 128u * KC * 2 + (size_t)NDIG * Np * (b_all ? Kp : KC) * 2 + 2 * 128 * 4 +
           2 * 128 * 4 + sizeof(FxBars) + 16;
}

// CTAs per SM (TMEM: na Npp columns rounded to a power of two, from 512), staging buffers
// (two when they fit the per-CTA share of the SM's 228 KB, 1 KB reserved per CTA) and the
// dynamic shared memory, at least 1/(ctas + 1) of the SM so that no further CTA co-resides
// (its TMEM allocation would wait for a CTA to finish all of its work)
struct FxCfg {
    int cols, ctas, nstg, b_all, tsets;
    size_t smem;
};
// tsets = 2 asks for two accumulator sets (one CTA per SM for 6 x 32 columns); it falls back
// to one set when they do not fit the 512 TMEM columns or the operator is not resident
static FxCfg fx_cfg(int dir, int N, int tsets = 1) {
    const int na = NACC;
    int Np, Kp, KC;
    fx_geometry(N, &Np, &Kp, &KC);
    FxCfg c;
    const int Npp = Np > 64 ? 64 : Np;
    if (tsets == 2 && 2 * na * Npp > 512) tsets = 1;
    c.tsets = tsets;
    const int need = tsets * na * Npp;
    c.cols = need <= 32 ? 32 : (need <= 64 ? 64 : (need <= 128 ? 128 : (need <= 256 ? 256 : 512)));
    c.ctas = c.cols <= 256 ? 2 : 1;
    size_t share = 233472 / c.ctas - 1024;
    const size_t stg = fx_stg_bytes(dir, N);
    c.b_all = stg + fx_rest_bytes(N, 1) <= share;
    if (!c.b_all && c.ctas == 2) {  // try one CTA per SM with all chunks resident
        c.ctas = 1;
        share = 233472 - 1024;
        c.b_all = stg + fx_rest_bytes(N, 1) <= share;
    }
    if (c.tsets == 2 && !c.b_all) return fx_cfg(dir, N, 1);
    const size_t rest = fx_rest_bytes(N, c.b_all);
    c.nstg = 2 * stg + rest <= share ? 2 : 1;
    const size_t b = c.nstg * stg + rest;
    const size_t floor_ = 233472 / (c.ctas + 1) + 1;
    c.smem = b > floor_ ? b : floor_;
    return c;
}

static size_t fx_smem_max(int dir) {
    size_t mx = 0;
    for (int n = 2; n <= 128; n++)
        for (int ts = 1; ts <= 2; ts++) {
            const size_t b = fx_cfg(dir, n, ts).smem;
            mx = b > mx ? b : mx;
        }
    return mx;
}

// ---- tuning table: accumulator sets per (direction, nodes, kind) class (kind 0 derivative,
// 1 filter), chosen by the autotuner (grmhd_tune_contractions) or read from a tuning file;
// 0 = not tuned (one set)
namespace {
std::mutex g_tune_lock;
std::map<std::tuple<int, int, int>, int> g_tune;
}  // namespace

void fx_tune_set(int dir, int N, int kind, int tsets) {
    std::lock_guard<std::mutex> lk(g_tune_lock);
    g_tune[std::make_tuple(dir, N, kind)] = tsets;
}

int fx_tune_get(int dir, int N, int kind) {
    std::lock_guard<std::mutex> lk(g_tune_lock);
    auto it = g_tune.find(std::make_tuple(dir, N, kind));
    return it == g_tune.end() ? 0 : it->second;
}

bool fx_two_sets_possible(int dir, int N) {
    if (!fx_supported(dir, N)) return false;
    return fx_cfg(dir, N, 2).tsets == 2;
}

template <int DIR, int WC, int WE>
static cudaError_t set_attr_fx() {
    return cudaFuncSetAttribute(k_contract_fx<DIR, WC, WE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)fx_smem_max(DIR));
}

template <int DIR>
static cudaError_t set_attr_fx_dir() {
    cudaError_t e;
    if ((e = set_attr_fx<DIR, 4, 4>()) != cudaSuccess) return e;
    return set_attr_fx<DIR, 8, 8>();
}

cudaError_t fx_init() {
    cudaError_t e;
    if ((e = set_attr_fx_dir<0>()) != cudaSuccess) return e;
    if ((e = set_attr_fx_dir<1>()) != cudaSuccess) return e;
    return set_attr_fx_dir<2>();
}

cudaError_t launch_contract_fx(int dir, const Dims& d, const DerivJob* jobs, int njobs, const uint8_t* img,
                               long long img_estride, int* err, cudaStream_t s, int stall, int kind, int tsets) {
    if (njobs <= 0) return cudaSuccess;
    if (kind != 0 && kind != 1) return cudaErrorNotSupported;
    const int N = dir == 0 ? d.Nr : (dir == 1 ? d.Nt : d.Np);
    if (!fx_supported(dir, N)) return cudaErrorNotSupported;
    // r and theta tiles are staged with bulk copies of row segments: 16-byte alignment
    // needs an even number of phi lines per row
    if (dir < 2 && (d.Np % 2)) return cudaErrorNotSupported;
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
    fp.npass = Np / fp.Npp;
    if (tsets <= 0) tsets = fx_tune_get(dir, N, kind);
    const FxCfg cfg = fx_cfg(dir, N, tsets == 2 ? 2 : 1);
    fp.tmem_cols = cfg.cols;
    fp.nstg = cfg.nstg;
    fp.b_all = cfg.b_all;
    fp.njobs = njobs;
    fp.stg_bytes = fx_stg_bytes(dir, N);
    fp.err = err;
    fp.stall = stall;
    fp.tsets = cfg.tsets;
    if (d.P >= (1LL << 31) || (d.P / 16 + d.E) * 2 * (long long)njobs >= (1LL << 31))
        return cudaErrorNotSupported;   // 32-bit line and item arithmetic
    fp.tpe = (uint32_t)((d.NtNp + 127) / 128);
    fp.nlf = dir == 1 ? (uint32_t)((long long)d.E * d.Nr * d.Np) : (uint32_t)(d.P / N);
    if (dir == 0) fp.ntiles = (long long)d.E * fp.tpe;
    else fp.ntiles = ((long long)fp.nlf + 127) / 128;
    if (fp.ntiles <= 0) return cudaSuccess;
    fp.per_job = (uint32_t)(fp.ntiles * fp.npass);
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long nitems = fp.ntiles * fp.npass * njobs;
    const long long grid = nitems < (long long)cfg.ctas * nsm ? nitems : (long long)cfg.ctas * nsm;
    const size_t sm = cfg.smem;
    // one CTA per SM: eight converter and eight epilogue warps (the register file holds
    // them at up to 112 registers a thread); two: four of each (96 registers)
    const bool w8 = cfg.ctas == 1;
    const unsigned nt = (unsigned)(w8 ? fx_threads(8, 8) : fx_threads(4, 4));
    if (dir == 0) {
        if (w8) k_contract_fx<0, 8, 8><<<(unsigned)grid, nt, sm, s>>>(d, fp);
        else k_contract_fx<0, 4, 4><<<(unsigned)grid, nt, sm, s>>>(d, fp);
    } else if (dir == 1) {
        if (w8) k_contract_fx<1, 8, 8><<<(unsigned)grid, nt, sm, s>>>(d, fp);
        else k_contract_fx<1, 4, 4><<<(unsigned)grid, nt, sm, s>>>(d, fp);
    } else {
        if (w8) k_contract_fx<2, 8, 8><<<(unsigned)grid, nt, sm, s>>>(d, fp);
        else k_contract_fx<2, 4, 4><<<(unsigned)grid, nt, sm, s>>>(d, fp);
    }
    return cudaGetLastError();
}

}  // namespace gk
