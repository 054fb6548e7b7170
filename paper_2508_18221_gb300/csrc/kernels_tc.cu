// Tensor-core spectral contractions for the mixed-precision modes (tcgen05, sm_103a).
//
// out[line][i] = scale * sum_j D[i][j] u[line][j] is a GEMM with M = lines (128 per CTA),
// N = output nodes, K = input nodes (the paper's derivative operators as matrices).
//   precision 1 (split BF16 x3): u (FP64 or FP32) and D are each split into three BF16
//     slices, x = x1 + x2 + x3, and the six products with slice-order sum <= 4
//     (a3 D1, a2 D2, a1 D3, a2 D1, a1 D2, a1 D1, smallest first) accumulate in FP32 in
//     tensor memory: about 24 significant bits, the accuracy of an FP32 contraction.
//   precision 2 (TF32): one kind::tf32 product of the FP32 values.
// Operands sit in shared memory in the K-major, non-swizzled core-matrix layout
// (8 rows x 16 bytes per core matrix; leading-byte offset = next core matrix along K,
// stride-byte offset = next 8-row group).  The operator image is prepared once on the
// host in exactly that layout and copied with one cp.async.bulk per CTA; the line tile
// is converted and split by the CTA's threads.  One thread issues the MMAs and commits
// them to an mbarrier; every wait is bounded and reports a timeout through *err.
#include <cuda_bf16.h>
#include <stdint.h>

#include "fp_convert.cuh"
#include "grmhd_internal.h"

namespace gk {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // tcgen05 descriptor version
    return d;                // base offset 0, relative LBO, no swizzle
}

// instruction descriptor: D = F32; A = B = BF16 (kind::f16) or TF32 (kind::tf32); both
// operands K-major; N >> 3 at bit 17, M >> 4 at bit 24
__device__ __forceinline__ uint32_t instr_desc(int tf32, int m, int n) {
    uint32_t ab = tf32 ? 2u : 1u;
    return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// byte offset of element (row, k) in a K-major non-swizzled tile; es = element bytes
__device__ __forceinline__ uint32_t core_off(int row, int k, int kcores, int es) {
    const int per = 16 / es;
    return (uint32_t)(((row >> 3) * kcores + k / per) * 128 + (row & 7) * 16 + (k % per) * es);
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
    uint32_t done = 0;
    // 2^16 tries, each parking the warp up to 20 us (about 1.3 s in all)
    for (int it = 0; it < (1 << 16) && !done; it++)
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
                     "selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(smem_u32(bar)), "r"(phase), "r"(20000u) : "memory");
    return done != 0;
}

__device__ __forceinline__ float to_f32(double x) { return d2f_rn(x); }
__device__ __forceinline__ float to_f32(float x) { return x; }

__device__ __forceinline__ void mma_issue(int tf32, uint32_t tmem, uint64_t da, uint64_t db, uint32_t id,
                                          uint32_t acc) {
    if (tf32)
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                     "l"(da), "l"(db), "r"(id), "r"(acc));
    else
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                     "l"(da), "l"(db), "r"(id), "r"(acc));
}

}  // namespace

// Shared-memory plan (bytes): [A slices | B image | 2 mbarriers | tmem address]
//   A: nsl x 128 x Kp x es,  B: nsl x Np x Kp x es  (nsl = 3 for BF16 x3, 1 for TF32)
template <int DIR, typename TIn>
__global__ void __launch_bounds__(128) k_contract_tc(Dims d, const TcJob* __restrict__ jobs,
                                                     const uint8_t* __restrict__ op_img, int N,
                                                     int Np, int Kp, int tf32, int tmem_cols,
                                                     const double* __restrict__ r_scale,
                                                     int* __restrict__ err) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const int es = tf32 ? 4 : 2;
    const int nsl = tf32 ? 1 : 3;
    const int kcores = Kp * es / 16;
    const uint32_t a_bytes = 128u * Kp * es;
    const uint32_t b_bytes = (uint32_t)Np * Kp * es;
    uint8_t* sA = sm;
    uint8_t* sB = sm + nsl * a_bytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + nsl * b_bytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);
    const int tid = threadIdx.x, warp = tid >> 5;
    const TcJob job = jobs[blockIdx.y];

    long long nlines, stride;
    if (DIR == 0) { nlines = (long long)d.E * d.NtNp; stride = d.NtNp; }
    else if (DIR == 1) { nlines = (long long)d.E * d.Nr * d.Np; stride = d.Np; }
    else { nlines = d.P / N; stride = 1; }
    const long long t0 = (long long)blockIdx.x * 128;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    // operator image: one bulk copy, completion counted in bytes on bars[0]
    if (tid == 0) {
        const uint32_t bytes = nsl * b_bytes;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bars[0])),
                     "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_u32(sB)),
                     "l"(op_img), "r"(bytes), "r"(smem_u32(&bars[0]))
                     : "memory");
    }
    // line tile: convert and split into the K-major layout (zero padding in K and lines).
    // Each thread first issues LD independent global loads, then converts them, so that
    // LD loads per thread are in flight at once (128 * Kp is a multiple of 128 * LD): 16 along
    // phi (a thread's loads lie along one line; measured -12 % per step against 8), 8 along r
    // and theta (16 measured +3 % on r, equal on theta).
    const int K = N;
    constexpr int LD = DIR == 2 ? 16 : 8;
    for (int base_idx = 0; base_idx < 128 * Kp; base_idx += 128 * LD) {
        TIn raw[LD];
#pragma unroll
        for (int u = 0; u < LD; u++) {
            const int idx = base_idx + u * 128 + tid;
            int m, k;
            if (DIR == 2) { m = idx / Kp; k = idx % Kp; }   // consecutive threads along a line
            else { k = idx / 128; m = idx % 128; }          // consecutive threads across lines
            const long long t = t0 + m;
            raw[u] = TIn(0);
            if (k < K && t < nlines) {
                long long base;
                if (DIR == 0) { long long e = t / d.NtNp; base = e * d.elem + (t - e * d.NtNp); }
                else if (DIR == 1) { long long eil = t / d.Np; base = eil * d.NtNp + (t - eil * d.Np); }
                else base = t * N;
                raw[u] = static_cast<const TIn*>(job.src)[base + (long long)k * stride];
            }
        }
        // all LD loads are issued before the first conversion
#pragma unroll
        for (int u = 0; u < LD; u++) {
            const int idx = base_idx + u * 128 + tid;
            int m, k;
            if (DIR == 2) { m = idx / Kp; k = idx % Kp; }
            else { k = idx / 128; m = idx % 128; }
            const uint32_t off = core_off(m, k, kcores, es);
            const float v = to_f32(raw[u]);
            if (tf32) {
                uint32_t w;
                asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(w) : "f"(v));
                *reinterpret_cast<uint32_t*>(sA + off) = w;
            } else {
                __nv_bfloat16 x1 = __float2bfloat16_rn(v);
                float r1 = v - __bfloat162float(x1);
                __nv_bfloat16 x2 = __float2bfloat16_rn(r1);
                __nv_bfloat16 x3 = __float2bfloat16_rn(r1 - __bfloat162float(x2));
                *reinterpret_cast<__nv_bfloat16*>(sA + off) = x1;
                *reinterpret_cast<__nv_bfloat16*>(sA + a_bytes + off) = x2;
                *reinterpret_cast<__nv_bfloat16*>(sA + 2 * a_bytes + off) = x3;
            }
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    bool ok = true;
    if (tid == 0) {
        ok = mbar_wait(&bars[0], 0);
        if (ok) {
            const uint32_t id = instr_desc(tf32, 128, Np);
            const uint32_t lbo = 128u, sbo = (uint32_t)kcores * 128u;
            const int kstep = tf32 ? 8 : 16;                 // K per instruction
            // slice pairs (a, b), smallest contribution first
            const int pa[6] = {2, 1, 0, 1, 0, 0};
            const int pb[6] = {0, 1, 2, 0, 1, 0};
            const int npairs = tf32 ? 1 : 6;
            uint32_t acc = 0;
            for (int q = 0; q < npairs; q++) {
                const int ia = tf32 ? 0 : pa[q], ib = tf32 ? 0 : pb[q];
                for (int c = 0; c < Kp / kstep; c++) {
                    uint64_t da = smem_desc(smem_u32(sA + ia * a_bytes) + c * 256, lbo, sbo);
                    uint64_t db = smem_desc(smem_u32(sB + ib * b_bytes) + c * 256, lbo, sbo);
                    mma_issue(tf32, tmem, da, db, id, acc);
                    acc = 1;
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&bars[1])));
        } else {
            atomicExch(err, 1);
            // release bars[1] so that the other threads do not wait in vain
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bars[1])) : "memory");
        }
    }
    __syncwarp();
    ok = mbar_wait(&bars[1], 0);
    if (!ok && (tid & 31) == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    // epilogue: warp w owns lines 32w..32w+31 (TMEM lanes), 8 output columns at a time
    // (the radial Jacobian multiplies in FP32: one rounding more than forming the product in
    // FP64 before the cast, at most 2^-24 relative, where the FP64 product kept the FP64
    // pipe 63-76 % busy in the radial instances)
    const int m = warp * 32 + (tid & 31);
    const long long t = t0 + m;
    long long base = 0;
    float scale = 1.0f;
    if (t < nlines) {
        if (DIR == 0) {
            long long e = t / d.NtNp;
            base = e * d.elem + (t - e * d.NtNp);
            if (r_scale) scale = d2f_rn(r_scale[e]);
        } else if (DIR == 1) { long long eil = t / d.Np; base = eil * d.NtNp + (t - eil * d.Np); }
        else base = t * N;
    }
    for (int cb = 0; cb < Np; cb += 8) {
        uint32_t r[8];
        uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb;
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                       "=r"(r[7])
                     : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (ok && t < nlines) {
            if (DIR == 2 && cb + 8 <= N && (N & 3) == 0) {
                // a line's 8 outputs are contiguous: two 16-byte stores
                float o[8];
#pragma unroll
                for (int j = 0; j < 8; j++) o[j] = __fmul_rn(scale, __uint_as_float(r[j]));
                float4* p4 = reinterpret_cast<float4*>(job.dst + base + cb);
                float4 lo = make_float4(o[0], o[1], o[2], o[3]), hi = make_float4(o[4], o[5], o[6], o[7]);
                if (job.accumulate) {
                    float4 a0 = p4[0], a1 = p4[1];
                    lo.x += a0.x; lo.y += a0.y; lo.z += a0.z; lo.w += a0.w;
                    hi.x += a1.x; hi.y += a1.y; hi.z += a1.z; hi.w += a1.w;
                }
                p4[0] = lo;
                p4[1] = hi;
            } else {
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    int i = cb + j;
                    if (i < N) {
                        float o = __fmul_rn(scale, __uint_as_float(r[j]));
                        float* p = job.dst + base + (long long)i * stride;
                        if (job.accumulate) *p += o;
                        else *p = o;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

size_t tc_smem_bytes(int N, int tf32) {
    const int es = tf32 ? 4 : 2, nsl = tf32 ? 1 : 3;
    const int Kp = (N + 15) / 16 * 16, Np = Kp;
    return (size_t)nsl * (128u * Kp * es + (size_t)Np * Kp * es) + 2 * sizeof(uint64_t) + 16;
}

template <int DIR, typename TIn>
static cudaError_t launch_dir(const Dims& d, const TcJob* jobs, int njobs, const uint8_t* img, int N,
                              int tf32, const double* r_scale, int* err, cudaStream_t s) {
    const int Kp = (N + 15) / 16 * 16, Np = Kp;
    const int cols = Np <= 32 ? 32 : (Np <= 64 ? 64 : (Np <= 128 ? 128 : 256));
    long long nlines = DIR == 0 ? (long long)d.E * d.NtNp : (DIR == 1 ? (long long)d.E * d.Nr * d.Np : d.P / N);
    long long nb = (nlines + 127) / 128;
    size_t sm = tc_smem_bytes(N, tf32);
    k_contract_tc<DIR, TIn><<<dim3((unsigned)nb, (unsigned)njobs), 128, sm, s>>>(d, jobs, img, N, Np, Kp, tf32, cols,
                                                                                 r_scale, err);
    return cudaGetLastError();
}

template <int DIR, typename TIn>
static cudaError_t set_attr() {
    return cudaFuncSetAttribute(k_contract_tc<DIR, TIn>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tc_smem_bytes(128, 0));
}

cudaError_t tc_init() {
    cudaError_t e;
    if ((e = set_attr<0, double>()) != cudaSuccess) return e;
    if ((e = set_attr<1, double>()) != cudaSuccess) return e;
    if ((e = set_attr<2, double>()) != cudaSuccess) return e;
    if ((e = set_attr<0, float>()) != cudaSuccess) return e;
    if ((e = set_attr<1, float>()) != cudaSuccess) return e;
    return set_attr<2, float>();
}

cudaError_t launch_contract_tc(int dir, int in_fp32, const Dims& d, const TcJob* jobs, int njobs,
                               const uint8_t* op_img, int tf32, const double* r_scale, int* err,
                               cudaStream_t s) {
    if (njobs <= 0) return cudaSuccess;
    const int N = dir == 0 ? d.Nr : (dir == 1 ? d.Nt : d.Np);
    if (N > 128) return cudaErrorNotSupported;
    if (in_fp32) {
        if (dir == 0) return launch_dir<0, float>(d, jobs, njobs, op_img, N, tf32, r_scale, err, s);
        if (dir == 1) return launch_dir<1, float>(d, jobs, njobs, op_img, N, tf32, nullptr, err, s);
        return launch_dir<2, float>(d, jobs, njobs, op_img, N, tf32, nullptr, err, s);
    }
    if (dir == 0) return launch_dir<0, double>(d, jobs, njobs, op_img, N, tf32, r_scale, err, s);
    if (dir == 1) return launch_dir<1, double>(d, jobs, njobs, op_img, N, tf32, nullptr, err, s);
    return launch_dir<2, double>(d, jobs, njobs, op_img, N, tf32, nullptr, err, s);
}

}  // namespace gk
