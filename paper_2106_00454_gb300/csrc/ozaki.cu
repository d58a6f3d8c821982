// ozaki.cu -- batched FP64-accurate matrix products on the BF16 tensor cores.
//
// The refinement products of the mixed path (H X, X^T Y, X^T X, X (I + E))
// need full FP64 accuracy, and GB300 issues FP64 at 1/58 of its FP32 rate.
// Ozaki's error-free splitting (Ozaki, Ogita, Oishi, Rump 2012) turns one
// FP64 product into a few exact low-precision ones:
//   * every row of the left operand and every column of the right one is
//     scaled by a power of two (2^e = the smallest power above its largest
//     magnitude), rounded to 47 bits and cut into P = 6 balanced digits of 8
//     bits: v / 2^e = sum_p d_p 2^{-8(p+1)+1}, d_1..d_5 in [-128, 127] and
//     |d_0| <= 129 -- all exact in BF16;
//   * the product of two digit slices is a sum of integer products of
//     magnitude < 2^15, so an FP32 tensor-core accumulation over a bounded k
//     range stays an exact integer (ozaki_tc.cu: the pairs of one weight over
//     128 k);
//   * C_ij = 2^{e_i + f_j} sum_{p+q <= P-1} 2^{-8(p+q+2)+2} (A_p B_q)_ij,
//     accumulated exactly in int64 and rounded once to FP64 (the 15 dropped
//     pairs weigh at most 2^-62 each).
// The error is dominated by the 47-bit rounding, |dC_ij| <~ 2^-48 (2^{e_i}
// sum_k |B_kj| + 2^{f_j} sum_k |A_ik|), ~4e-15 relative to the row and column
// scales.  The slices are stored k-contiguous ([p][vector][k],
// k padded to a multiple of 32) for both operands: K-major tiles for the
// tensor-core kernel of ozaki_tc.cu.
#include <cuda_bf16.h>
#include <math.h>

#include "wpcd_internal.cuh"

namespace wpcd {

constexpr int kOzP = kOzDigits;  // slices per operand
constexpr int kOzKC = 32;  // k staged per step

int oz_kpad(int n) { return (n + kOzKC - 1) / kOzKC * kOzKC; }
size_t oz_slice_elems(int n) { return (size_t)kOzP * n * oz_kpad(n); }

// GB300 issues FP64 at 2 operations per clock per SM, so the split works on
// the IEEE-754 fields with integer operations.
//
// N = rint(x 2^{47-e}) for |x| < 2^e (round half to even): x = m 2^{E-1075}
// with the 53-bit significand m, so N = m 2^{-s}, s = 1028 + e - E >= 6.
__device__ __forceinline__ long long oz_scaled(double x, int e)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    if (E == 0 || E == 0x7FF) {  // zero, subnormal or not finite: the FP64 route
        if ((b << 1) == 0) return 0;
        return __double2ll_rn(ldexp(x, 47 - e));
    }
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int s = 1028 + e - E;
    unsigned long long q = 0;
    if (s < 54) {  // for s >= 54, m 2^{-s} < 1/2
        q = m >> s;
        const unsigned long long rem = m & ((1ull << s) - 1), half = 1ull << (s - 1);
        q += (rem > half || (rem == half && (q & 1))) ? 1 : 0;
    }
    return (b >> 63) ? -(long long)q : (long long)q;
}

// BF16 bits of a small integer (|d| < 2^8, exact): 1.5 2^23 + d as an FP32 bit
// pattern, minus 1.5 2^23, leaves d in FP32 with a zero low half.
__device__ __forceinline__ __nv_bfloat16 oz_bf16_of_int(int d)
{
    const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;
    return __ushort_as_bfloat16((unsigned short)(__float_as_uint(f) >> 16));
}

// The six balanced 8-bit digits of x / 2^e: N = rint(x 2^{47-e}) (|N| <= 2^47),
// then N = d0 2^40 + d1 2^32 + ... + d5 with d1..d5 in [-128, 127] and
// |d0| <= 129 -- all exact in BF16, every digit product below 2^15 in
// magnitude, and the signs of the truncated lower products vary, so their
// sum grows like sqrt(k) instead of k.
__device__ __forceinline__ void oz_digit_set(long long N, int *d)
{
    // the three low digits from the low 24 bits (unsigned), their carry into
    // the high part, then the three high digits: 32-bit operations only
    int t = (int)((unsigned)N & 0xFFFFFFu), hi = (int)(N >> 24);
#pragma unroll
    for (int p = kOzP - 1; p >= 3; --p) {
        d[p] = ((t + 128) & 0xFF) - 128;
        t = (t - d[p]) >> 8;  // exact: t - d is a multiple of 256
    }
    hi += t;  // the carry, 0 or 1
#pragma unroll
    for (int p = 2; p >= 1; --p) {
        d[p] = ((hi + 128) & 0xFF) - 128;
        hi = (hi - d[p]) >> 8;
    }
    d[0] = hi;
}

// Two neighbouring elements (k, k + 1) of one vector: their digits as BF16
// pairs, one 32-bit store per digit plane.
__device__ __forceinline__ void oz_digits2(double x0, double x1, int e, __nv_bfloat16 *d, size_t stride)
{
    int a[kOzP], b[kOzP];
    oz_digit_set(oz_scaled(x0, e), a);
    oz_digit_set(oz_scaled(x1, e), b);
#pragma unroll
    for (int p = 0; p < kOzP; ++p) {
        __nv_bfloat162 v;
        v.x = oz_bf16_of_int(a[p]);
        v.y = oz_bf16_of_int(b[p]);
        *reinterpret_cast<__nv_bfloat162 *>(d + (size_t)p * stride) = v;
    }
}

// Magnitude of x as an ordered integer (the IEEE-754 bits without the sign).
__device__ __forceinline__ unsigned long long oz_mag(double x)
{
    return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// e with max|v| < 2^e from the magnitude bits of the largest |v| (0 for an
// all-zero vector): 2^{E-1023} <= max < 2^{E-1022}.
__device__ __forceinline__ int oz_exp_of(unsigned long long mag)
{
    const int E = (int)(mag >> 52);
    if (E != 0) return E - 1022;
    int ex = 0;
    if (mag != 0) frexp(__longlong_as_double((long long)mag), &ex);  // subnormal
    return ex;
}

// Row slices: S[b][p][v][k] = digit p of M[v][k], one warp per row v.  The
// row is read once into registers (lane l holds the pairs k = 2 l + 64 j,
// k + 1, all loads issued before any is used), its exponent comes from a warp
// maximum, and the digits are written from the registers with k fastest
// (coalesced); k in [n, Kp) is zero padding.
// PAIRS per lane: Kp <= 64 PAIRS (the launch picks the smallest of 4, 8, 16).
template <int PAIRS>
__global__ void __launch_bounds__(256) k_oz_split_rows(int n, int Kp, const double *M_all, int *e_all,
                                                       __nv_bfloat16 *S_all)
{
    constexpr int kOzRowPairs = PAIRS;
    const int b = blockIdx.y, v = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (v >= n) return;
    const double *row = M_all + (size_t)b * n * n + (size_t)v * n;
    double x0[kOzRowPairs], x1[kOzRowPairs];
    unsigned long long m = 0;
#pragma unroll
    for (int j = 0; j < kOzRowPairs; ++j) {
        const int k = 2 * lane + 64 * j;
        x0[j] = k < n ? row[k] : 0.0;
        x1[j] = k + 1 < n ? row[k + 1] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < kOzRowPairs; ++j) m = max(m, max(oz_mag(x0[j]), oz_mag(x1[j])));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int ex = oz_exp_of(m);
    if (lane == 0) e_all[(size_t)b * n + v] = ex;
    __nv_bfloat16 *S = S_all + (size_t)b * kOzP * n * Kp + (size_t)v * Kp;
#pragma unroll
    for (int j = 0; j < kOzRowPairs; ++j) {
        const int k = 2 * lane + 64 * j;  // Kp is even: pairs (k, k + 1)
        if (k < Kp) oz_digits2(x0[j], x1[j], ex, S + k, (size_t)n * Kp);
    }
}

// Column slices for Kp <= kOzColBlockKp: one CTA (32 x 8) per 32 columns reads
// its Kp x 32 block once into shared memory (pitch 33 doubles; v fastest,
// coalesced), takes the column maxima while loading, and writes the digits
// from shared memory along k (two per thread, coalesced).
constexpr int kOzColBlockKp = 384;  // 101 KB of shared memory at most
__global__ void __launch_bounds__(256) k_oz_split_cols_block(int n, int Kp, const double *M_all, int *e_all,
                                                             __nv_bfloat16 *S_all)
{
    extern __shared__ double blk[];  // [Kp][33]
    __shared__ unsigned long long mcol[8][32];
    __shared__ int ecol[32];
    const int b = blockIdx.y;
    const int v0 = blockIdx.x * 32, tx = threadIdx.x, ty = threadIdx.y, v = v0 + tx;
    const double *M = M_all + (size_t)b * n * n;
    unsigned long long m = 0;
#pragma unroll 8
    for (int k = ty; k < Kp; k += 8) {
        const double x = (k < n && v < n) ? M[(size_t)k * n + v] : 0.0;
        blk[k * 33 + tx] = x;
        m = max(m, oz_mag(x));
    }
    mcol[ty][tx] = m;
    __syncthreads();
    if (ty == 0) {
        for (int r = 1; r < 8; ++r) m = max(m, mcol[r][tx]);
        ecol[tx] = oz_exp_of(m);
        if (v < n) e_all[(size_t)b * n + v] = ecol[tx];
    }
    __syncthreads();
    __nv_bfloat16 *S = S_all + (size_t)b * kOzP * n * Kp;
    for (int r = ty; r < 32 && v0 + r < n; r += 8)  // column v0 + r, k pairs 2 tx + 64 j
        for (int k = 2 * tx; k < Kp; k += 64)
            oz_digits2(blk[k * 33 + r], blk[(k + 1) * 33 + r], ecol[r], S + (size_t)(v0 + r) * Kp + k,
                       (size_t)n * Kp);
}

// Column slices for larger Kp: S[b][p][v][k] = digit p of M[k][v], one CTA
// (32 x 8) per 32 columns: the column maxima first (reads along v), then 64 x 32 tiles
// transposed through shared memory so that both the reads (v fastest) and the
// writes (k fastest, two per thread) are coalesced.
__global__ void __launch_bounds__(256) k_oz_split_cols(int n, int Kp, const double *M_all, int *e_all,
                                                       __nv_bfloat16 *S_all)
{
    __shared__ double tile[64][33];
    __shared__ unsigned long long mcol[8][32];
    __shared__ int ecol[32];
    const int b = blockIdx.y;
    const int v0 = blockIdx.x * 32, tx = threadIdx.x, ty = threadIdx.y;
    const double *M = M_all + (size_t)b * n * n;
    unsigned long long m = 0;
    if (v0 + tx < n)
        for (int k = ty; k < n; k += 8) m = max(m, oz_mag(M[(size_t)k * n + v0 + tx]));
    mcol[ty][tx] = m;
    __syncthreads();
    if (ty == 0) {
        for (int r = 1; r < 8; ++r) m = max(m, mcol[r][tx]);
        ecol[tx] = oz_exp_of(m);
        if (v0 + tx < n) e_all[(size_t)b * n + v0 + tx] = ecol[tx];
    }
    __syncthreads();
    __nv_bfloat16 *S = S_all + (size_t)b * kOzP * n * Kp;
    for (int k0 = 0; k0 < Kp; k0 += 64) {  // 64 k x 32 v per tile, read along v
        for (int r = ty; r < 64; r += 8) {
            const int k = k0 + r, v = v0 + tx;
            tile[r][tx] = (k < n && v < n) ? M[(size_t)k * n + v] : 0.0;
        }
        __syncthreads();
        for (int r = ty; r < 32; r += 8) {  // column v0 + r, k pair k0 + 2 tx: written along k
            const int v = v0 + r, k = k0 + 2 * tx;
            if (v < n && k < Kp) oz_digits2(tile[2 * tx][r], tile[2 * tx + 1][r], ecol[r], S + (size_t)v * Kp + k, (size_t)n * Kp);
        }
        __syncthreads();
    }
}

// Digit slices of the rows (cols = false) or columns (cols = true) of `items`
// n x n matrices: S [items][P][n][Kp] bf16, e [items][n].
cudaError_t launch_oz_split(int n, int items, bool cols, const double *M, __nv_bfloat16 *S, int *e, cudaStream_t st)
{
    const int Kp = oz_kpad(n);
    if (!cols) {
        const dim3 g((n + 7) / 8, items);
        if (Kp <= 256) k_oz_split_rows<4><<<g, 256, 0, counted(st)>>>(n, Kp, M, e, S);
        else if (Kp <= 512) k_oz_split_rows<8><<<g, 256, 0, counted(st)>>>(n, Kp, M, e, S);
        else k_oz_split_rows<16><<<g, 256, 0, counted(st)>>>(n, Kp, M, e, S);
    } else if (Kp <= kOzColBlockKp) {
        const size_t smem = (size_t)Kp * 33 * sizeof(double);
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_oz_split_cols_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kOzColBlockKp * 33 * (int)sizeof(double));
        k_oz_split_cols_block<<<dim3((n + 31) / 32, items), dim3(32, 8), smem, counted(st)>>>(n, Kp, M, e, S);
    } else {
        k_oz_split_cols<<<dim3((n + 31) / 32, items), dim3(32, 8), 0, counted(st)>>>(n, Kp, M, e, S);
    }
    return cudaGetLastError();
}

// C = A B from the row slices of A and the column slices of B.
cudaError_t launch_oz_gemm_slices(int n, int items, const __nv_bfloat16 *sa, const int *ea, const __nv_bfloat16 *sb,
                                  const int *eb, double *C, cudaStream_t st, int digits, bool sym, int *err,
                                  int a_items)
{
    return launch_oz_gemm_tc(n, items, sa, ea, sb, eb, C, digits, sym, err, st, a_items);
}

// C = op(A) B for `items` n x n FP64 matrices (op(A) = A^T when ta), through
// the slices.  Scratch: sa, sb hold oz_slice_elems(n) bf16 per item; ea, eb n ints per item.
cudaError_t launch_oz_gemm(int n, int items, bool ta, const double *A, const double *B, double *C,
                           __nv_bfloat16 *sa, __nv_bfloat16 *sb, int *ea, int *eb, cudaStream_t st,
                           int *err)
{
    cudaError_t e;
    // rows of op(A): rows of A, or columns of A when transposed; columns of B
    if ((e = launch_oz_split(n, items, ta, A, sa, ea, st))) return e;
    if ((e = launch_oz_split(n, items, true, B, sb, eb, st))) return e;
    return launch_oz_gemm_slices(n, items, sa, ea, sb, eb, C, st, kOzP, false, err);
}

}  // namespace wpcd
