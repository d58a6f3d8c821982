// project_tc.cu -- (a1) reduced-precision projection: the angle integrals of
// the Yukawa radial forms as a contraction on the tensor cores.
//
// The projection's inner step (Sec. 3.2, Eq. "WP potential matrix identity",
// after the partial-wave expansion) is, for every fine pair (k_a, k_b) of a
// mesh and every mass m of the generator,
//     I_L[m](k_a, k_b) = 2 pi sum_x w_x P_L(x) F_m(x),
//     F_m(x) = 1 / ((k_a - k_b)^2 + 2 k_a k_b (1 - x) + m^2),
// a product of the matrix F [pairs x 96 angles] with the table
// w_x P_L(x) [96 x (L_max + 1)].  Here:
//   * F is evaluated in FP32 (the squared momentum transfer written as a sum
//     of non-negative terms, so there is no cancellation, with 1 - x taken
//     from the FP64 nodes);
//   * split-precision correction in the Ozaki manner: every row of F is scaled
//     by a power of two from its largest value (at the largest node x, where
//     the transfer is smallest), rounded to a 31-bit integer and cut into
//     four balanced 8-bit digits; every column of the table likewise, from
//     its own largest |value|.  Digits are exact in BF16 and a product of two
//     is at most 2^14, so the FP32 accumulator of one weight (at most four
//     digit pairs) over the 96 angles holds an exact integer (< 2^24): the
//     tensor core's accumulation adds no error;
//   * the ten digit pairs of weight p + q <= 3 (the dropped ones weigh
//     <= 2^-32) run as tcgen05.mma kind::f16 (BF16 operands, FP32
//     accumulation in tensor memory), M = 128 fine pairs, N = 16 (L <= 15),
//     K = 96 in three 32-k spans of the 64-byte-swizzled K-major layout, one
//     accumulator per (mass, weight); the epilogue assembles each integral in
//     FP64 from the exact integer sums and the two scales;
//   * the integrals leave as FP32 [pair][mass][16] (their FP32 rounding,
//     2^-24, is below the evaluation error of F); the potential terms and the
//     bin reduction that use them stay FP64 (k_project in mesh_project.cu).
// One CTA per tile of 128 consecutive fine pairs (pair = bin pair * Q^2 +
// qa Q + qb, bin pairs (i <= j) of the upper triangle).  Every wait on the
// tensor core is bounded; on a timeout the kernel records kDevTimeout and
// frees its tensor memory.
#include <cuda_bf16.h>
#include <stdint.h>

#include "potential.cuh"
#include "wpcd_internal.cuh"

namespace wpcd {

constexpr int kPtM = 128;                  // fine pairs per tile (TMEM lanes)
constexpr int kPtN = 16;                   // L = 0 .. 15 (columns per accumulator)
constexpr int kPtDigits = 4;               // balanced 8-bit digits per operand
constexpr int kPtSpans = kAngleQ / 32;     // 32-k spans of 64 bytes
constexpr int kPtASplit = kPtM * kAngleQ * 2;   // one BF16 term of A: 24 KB
constexpr int kPtBSplit = kPtN * kAngleQ * 2;   // one BF16 term of B: 3 KB
// alignment slack | A digits | B digits | barrier, TMEM slot | B in FP64 [16][96] | column exponents
constexpr int kPtSmem = 1024 + kPtDigits * (kPtASplit + kPtBSplit) + 64 + kPtN * kAngleQ * 8 + kPtN * 4 + 64;
constexpr int kPtThreads = 256;
constexpr int kPtTmemCols = 256;           // 3 masses x 4 weights x 16 columns, allocated as a power of two
constexpr long long kPtWaitCycles = 1ll << 31;
// D F32, A and B BF16, both K-major, N = 16, M = 128 (the encoding of the digit products)
constexpr uint32_t kPtIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kPtN >> 3) << 17) |
                              ((uint32_t)(kPtM >> 4) << 24);

__device__ __forceinline__ uint32_t pt_smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (row r, k) in a K-major operand of 64-byte rows per
// 32-k span (span blocks of rows x 64 bytes), 64-byte swizzle: the 16-byte unit
// index within a row is XORed with bits 1-2 of the row.
__device__ __forceinline__ uint32_t pt_sw64(int r, int k, int rows)
{
    const int s = k >> 5, kk = k & 31;
    return (uint32_t)(s * rows * 64 + r * 64 + ((((kk >> 3) ^ (r >> 1)) & 3) << 4) + ((kk & 7) << 1));
}

__device__ __forceinline__ uint64_t pt_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;           // leading byte offset (unused inside a swizzle span)
    d |= (uint64_t)(512 >> 4) << 32;  // stride byte offset: 8 rows x 64 bytes
    d |= (uint64_t)1 << 46;           // descriptor version
    d |= (uint64_t)4 << 61;           // 64-byte swizzle
    return d;
}

__device__ __forceinline__ bool pt_try(uint32_t a, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ bool pt_wait(uint32_t a, uint32_t parity)
{
    const long long t0 = clock64();
    while (!pt_try(a, parity))
        if (clock64() - t0 > kPtWaitCycles) return false;
    return true;
}

// v = 2^(e - 30) (d0 2^24 + d1 2^16 + d2 2^8 + d3) to the nearest integer
// multiple of 2^(e - 30), |v| < 2^(e + 1): balanced digits d1..d3 in
// [-128, 127], |d0| <= 128, all exact in BF16; d[p] is digit p.
__device__ __forceinline__ void digits4(double v, int e, __nv_bfloat16 *d)
{
    long long N = llrint(ldexp(v, 30 - e));
#pragma unroll
    for (int p = kPtDigits - 1; p > 0; --p) {
        const long long r = ((N + 128) & 255) - 128;
        d[p] = __float2bfloat16_rn((float)r);
        N = (N - r) >> 8;
    }
    d[0] = __float2bfloat16_rn((float)N);
}

__global__ void __launch_bounds__(kPtThreads) k_angle_tc(const ChanDev *chans, const int *group, int N, int Q, int Lm,
                                                       const double *gp, const double *angx, const double *angw,
                                                       long long n_pairs, float *Iout, int *err)
{
    extern __shared__ unsigned char pt_raw[];
    const uint32_t raw_s = pt_smem_u32(pt_raw);
    const uint32_t base_s = (raw_s + 1023u) & ~1023u;  // the swizzle follows address bits
    unsigned char *base = pt_raw + (base_s - raw_s);
    unsigned char *As = base;                          // 4 digits x [3 spans][128 rows][64 B]
    unsigned char *Bs = base + kPtDigits * kPtASplit;  // 4 digits x [3 spans][16 rows][64 B]
    uint64_t *bar = reinterpret_cast<uint64_t *>(Bs + kPtDigits * kPtBSplit);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 1);
    double *Bd = reinterpret_cast<double *>(reinterpret_cast<unsigned char *>(bar) + 64);  // [16][96]
    int *eCol = reinterpret_cast<int *>(Bd + kPtN * kAngleQ);                              // [16]
    __shared__ float omx[kAngleQ];                 // 1 - x
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t bar_s = pt_smem_u32(bar);
    const long long pair0 = (long long)blockIdx.x * kPtM;

    // w_x P_L(x), split, into B (rows L, k = x); 1 - x in FP64 then FP32
    for (int x = tid; x < kAngleQ; x += kPtThreads) {
        const double xv = angx[x];
        omx[x] = (float)(1.0 - xv);
        double p0 = 1.0, p1 = xv;
        for (int L = 0; L < kPtN; ++L) {
            double pl;
            if (L == 0) pl = 1.0;
            else if (L == 1) pl = xv;
            else {
                pl = ((2.0 * L - 1.0) * xv * p1 - (L - 1.0) * p0) / L;
                p0 = p1;
                p1 = pl;
            }
            Bd[L * kAngleQ + x] = L <= Lm ? 2.0 * kPi * angw[x] * pl : 0.0;
        }
    }
    __syncthreads();
    if (tid < kPtN) {  // column exponents: 2^e <= max_x |B[L][x]| < 2^(e + 1)
        double mx = 0.0;
        for (int x = 0; x < kAngleQ; ++x) mx = fmax(mx, fabs(Bd[tid * kAngleQ + x]));
        eCol[tid] = mx > 0.0 ? ilogb(mx) : 0;
    }
    __syncthreads();
    for (int e = tid; e < kPtN * kAngleQ; e += kPtThreads) {
        const int L = e / kAngleQ, x = e - L * kAngleQ;
        __nv_bfloat16 d[kPtDigits];
        digits4(Bd[e], eCol[L], d);
        const uint32_t o = pt_sw64(L, x, kPtN);
#pragma unroll
        for (int p = 0; p < kPtDigits; ++p) *reinterpret_cast<__nv_bfloat16 *>(Bs + p * kPtBSplit + o) = d[p];
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_s) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(pt_smem_u32(tmem_slot)),
                     "r"(kPtTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    // this thread's fine pair(s): rows r = tid & 127, angles x = (tid >> 7) + 2 j
    const double *kq = chans[group[0]].kq;  // the fine nodes of the group's mesh
    const int r = tid & (kPtM - 1), xh = tid >> 7;
    const long long pr = pair0 + r;
    float dd = 0.0f, s2 = 0.0f;
    if (pr < n_pairs) {
        const int QQ = Q * Q;
        const long long b = pr / QQ;
        const int w = (int)(pr - b * QQ), qa = w / Q, qb = w - qa * Q;
        int j = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
        while ((long long)(j + 1) * (j + 2) / 2 <= b) ++j;
        while ((long long)j * (j + 1) / 2 > b) --j;
        const int i = (int)(b - (long long)j * (j + 1) / 2);
        const double pp = kq[i * Q + qa], p = kq[j * Q + qb];
        dd = (float)(pp - p);
        s2 = (float)(2.0 * pp * p);
    }
    // the smallest 1 - x (the largest node) gives the largest F of a row
    float omin = omx[0];
    for (int x = 1; x < kAngleQ; ++x) omin = fminf(omin, omx[x]);
    bool ok = true;
    int erow[3];  // this row's exponent per mass (the epilogue threads hold their own rows)
    for (int m = 0; m < 3; ++m) {
        const float mm = (float)(gp[m] * gp[m]);
        if (m > 0) {  // the MMAs of the previous mass must be done with A
            ok = ok && pt_wait(bar_s, (uint32_t)((m - 1) & 1));
        }
        const int er = pr < n_pairs ? ilogb(__frcp_rn(fmaf(dd, dd, fmaf(s2, omin, mm)))) : 0;
        erow[m] = er;
        for (int x = xh; x < kAngleQ; x += 2) {
            float F = 0.0f;
            if (pr < n_pairs) F = __frcp_rn(fmaf(dd, dd, fmaf(s2, omx[x], mm)));
            __nv_bfloat16 d[kPtDigits];
            digits4((double)F, er, d);
            const uint32_t o = pt_sw64(r, x, kPtM);
#pragma unroll
            for (int p = 0; p < kPtDigits; ++p) *reinterpret_cast<__nv_bfloat16 *>(As + p * kPtASplit + o) = d[p];
        }
        // the generic-proxy stores become visible to the tensor core
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // digit pairs (p, q) of weight p + q <= 3, by weight: (0,0) | (0,1) (1,0) |
            // (0,2) (2,0) (1,1) | (0,3) (3,0) (1,2) (2,1), one nibble per pair; the pairs
            // of one weight share the accumulator (mass, weight)
            for (int t = 0; t < 10; ++t) {
                const int ta = (int)((0x2130120100ull >> (4 * t)) & 0xF), tb = (int)((0x1203102010ull >> (4 * t)) & 0xF);
                const bool first = t == 0 || t == 1 || t == 3 || t == 6;  // the first pair of each weight
                uint32_t acc = first ? 0u : 1u;
                const uint32_t dcol = tmem + (uint32_t)((m * kPtDigits + ta + tb) * kPtN);
                for (int s = 0; s < kPtSpans; ++s)
                    for (int kk = 0; kk < 2; ++kk) {  // K = 16 steps, 32 bytes apart inside a span
                        const uint32_t a_s = pt_smem_u32(As) + ta * kPtASplit + s * kPtM * 64 + kk * 32;
                        const uint32_t b_s = pt_smem_u32(Bs) + tb * kPtBSplit + s * kPtN * 64 + kk * 32;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dcol),
                            "l"(pt_desc(a_s)), "l"(pt_desc(b_s)), "r"(kPtIdesc), "r"(acc)
                            : "memory");
                        acc = 1;
                    }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_s)
                         : "memory");
        }
    }
    ok = ok && pt_wait(bar_s, 0u);  // the third mass (phase 2 has parity 0)
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!__syncthreads_and(ok ? 1 : 0)) {
        if (tid == 0) record_error(err, kDevTimeout);
    } else if (warp < 4) {
        // warp w reads TMEM lanes 32 w .. 32 w + 31 = rows of the tile (its own rows:
        // tid = row), per mass the four weight accumulators of 16 columns each
        const long long row = pair0 + tid;
        const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16);
        for (int m = 0; m < 3; ++m) {
            uint32_t v[16 * kPtDigits];
#pragma unroll
            for (int d = 0; d < kPtDigits; ++d) {
                uint32_t *u = v + 16 * d;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15}, [%16];"
                    : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
                      "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]),
                      "=r"(u[15])
                    : "r"(ta + (uint32_t)((m * kPtDigits + d) * kPtN)));
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < n_pairs) {
                float out[kPtN];
#pragma unroll
                for (int L = 0; L < kPtN; ++L) {
                    // exact integer sums of weights d = 0..3 times 2^(48 - 8 d), scaled back
                    double sum = 0.0;
#pragma unroll
                    for (int d = 0; d < kPtDigits; ++d) sum += ldexp((double)__uint_as_float(v[16 * d + L]), 48 - 8 * d);
                    out[L] = (float)ldexp(sum, erow[m] + eCol[L] - 60);
                }
                float4 *o = reinterpret_cast<float4 *>(Iout + (size_t)row * 48 + m * kPtN);
#pragma unroll
                for (int q = 0; q < 4; ++q) o[q] = make_float4(out[4 * q], out[4 * q + 1], out[4 * q + 2], out[4 * q + 3]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kPtTmemCols)
                     : "memory");
    }
}

size_t angle_tc_buffer_bytes(int N, int Q) { return (size_t)N * (N + 1) / 2 * Q * Q * 48 * sizeof(float); }

// Angle integrals of every fine pair of the mesh of chans[group[0]], for the
// three Yukawa masses gp[0..2] and L = 0..Lm (Lm <= 15): Iout [pair][3][16] FP32.
cudaError_t launch_angle_tc(const ChanDev *chans_dev, const int *group_dev, int N, int Q, int Lm, const double *gp_dev,
                            const double *angx, const double *angw, float *Iout, int *err, cudaStream_t st)
{
    if (Lm >= kPtN || N < 1 || Q < 1) return cudaErrorInvalidValue;
    const long long n_pairs = (long long)N * (N + 1) / 2 * Q * Q;
    const long long tiles = (n_pairs + kPtM - 1) / kPtM;
    if (tiles > 0x7fffffffll) return cudaErrorInvalidValue;
    cudaError_t e = raise_smem_limit((const void *)k_angle_tc, kPtSmem);
    if (e != cudaSuccess) return e;
    k_angle_tc<<<(unsigned)tiles, kPtThreads, kPtSmem, counted(st)>>>(chans_dev, group_dev, N, Q, Lm, gp_dev, angx,
                                                                     angw, n_pairs, Iout, err);
    return cudaGetLastError();
}

}  // namespace wpcd
