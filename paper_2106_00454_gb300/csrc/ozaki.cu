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

// Exponent of every row (COLS = false) or column (COLS = true) of the n x n
// matrices: e with max|v| < 2^e (0 for an all-zero vector).  For rows one warp
// per row, for columns one thread per column (both read coalesced).
template <bool COLS>
__global__ void k_oz_exp(int n, const double *M_all, int *e_all)
{
    const int b = blockIdx.y;
    const double *M = M_all + (size_t)b * n * n;
    double m = 0.0;
    int v;
    if (COLS) {
        v = blockIdx.x * blockDim.x + threadIdx.x;
        if (v >= n) return;
        for (int k = 0; k < n; ++k) m = fmax(m, fabs(M[(size_t)k * n + v]));
    } else {
        v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
        if (v >= n) return;
        for (int k = threadIdx.x & 31; k < n; k += 32) m = fmax(m, fabs(M[(size_t)v * n + k]));
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) != 0) return;
    }
    int ex = 0;
    if (m > 0.0) frexp(m, &ex);  // m < 2^ex
    e_all[(size_t)b * n + v] = ex;
}

// The six balanced 8-bit digits of x / 2^e: N = rint(x 2^{47-e}) (|N| <= 2^47),
// then N = d0 2^40 + d1 2^32 + ... + d5 with d1..d5 in [-128, 127] and
// |d0| <= 129 -- all exact in BF16, every digit product below 2^15 in
// magnitude, and the signs of the truncated lower products vary, so their
// sum grows like sqrt(k) instead of k.
__device__ __forceinline__ void oz_digits(double x, int e, __nv_bfloat16 *d, size_t stride)
{
    const int be = 1023 + 47 - e;  // biased exponent of 2^{47-e}
    const double scale = (be >= 1 && be <= 2046) ? __hiloint2double(be << 20, 0) : ldexp(1.0, 47 - e);  // exact
    long long N = __double2ll_rn(x * scale);
#pragma unroll
    for (int p = kOzP - 1; p >= 1; --p) {
        const long long dig = ((N + 128) & 0xFF) - 128;
        d[(size_t)p * stride] = __float2bfloat16_rn((float)(int)dig);
        N = (N - dig) >> 8;  // exact: N - dig is a multiple of 256
    }
    d[0] = __float2bfloat16_rn((float)(int)N);
}

// Row slices: S[b][p][v][k] = digit p of M[v][k]; one thread per element, k
// fastest (coalesced reads and writes); k in [n, Kp) is zero padding.
__global__ void k_oz_split_rows(int n, int Kp, const double *M_all, const int *e_all, __nv_bfloat16 *S_all)
{
    const int b = blockIdx.z, v = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Kp) return;
    const double x = (k < n) ? M_all[(size_t)b * n * n + (size_t)v * n + k] : 0.0;
    oz_digits(x, e_all[(size_t)b * n + v], S_all + (size_t)b * kOzP * n * Kp + (size_t)v * Kp + k, (size_t)n * Kp);
}

// Column slices: S[b][p][v][k] = digit p of M[k][v]; 32 x 32 tiles transposed
// through shared memory so that both the reads (v fastest) and the writes (k
// fastest) are coalesced.  Block 32 x 8.
__global__ void k_oz_split_cols(int n, int Kp, const double *M_all, const int *e_all, __nv_bfloat16 *S_all)
{
    __shared__ double tile[32][33];
    const int b = blockIdx.z;
    const int v0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    const double *M = M_all + (size_t)b * n * n;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int k = k0 + r, v = v0 + threadIdx.x;
        tile[r][threadIdx.x] = (k < n && v < n) ? M[(size_t)k * n + v] : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int v = v0 + r, k = k0 + threadIdx.x;
        if (v >= n || k >= Kp) continue;
        oz_digits(tile[threadIdx.x][r], e_all[(size_t)b * n + v],
                  S_all + (size_t)b * kOzP * n * Kp + (size_t)v * Kp + k, (size_t)n * Kp);
    }
}

// C = op(A) B for `items` n x n FP64 matrices (op(A) = A^T when ta), through
// the slices.  Scratch: sa, sb hold oz_slice_elems(n) bf16 per item; ea, eb n ints per item.
// Digit slices of the rows (cols = false) or columns (cols = true) of `items`
// n x n matrices: S [items][P][n][Kp] bf16, e [items][n].
cudaError_t launch_oz_split(int n, int items, bool cols, const double *M, __nv_bfloat16 *S, int *e, cudaStream_t st)
{
    const int Kp = oz_kpad(n);
    if (cols) {
        k_oz_exp<true><<<dim3((n + 127) / 128, items), 128, 0, st>>>(n, M, e);
        k_oz_split_cols<<<dim3((n + 31) / 32, (Kp + 31) / 32, items), dim3(32, 8), 0, st>>>(n, Kp, M, e, S);
    } else {
        k_oz_exp<false><<<dim3((n + 7) / 8, items), 256, 0, st>>>(n, M, e);
        k_oz_split_rows<<<dim3((Kp + 127) / 128, n, items), 128, 0, st>>>(n, Kp, M, e, S);
    }
    return cudaGetLastError();
}

// C = A B from the row slices of A and the column slices of B.
cudaError_t launch_oz_gemm_slices(int n, int items, const __nv_bfloat16 *sa, const int *ea, const __nv_bfloat16 *sb,
                                  const int *eb, double *C, cudaStream_t st, int digits, bool sym, int *err)
{
    return launch_oz_gemm_tc(n, items, sa, ea, sb, eb, C, digits, sym, err, st);
}

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
