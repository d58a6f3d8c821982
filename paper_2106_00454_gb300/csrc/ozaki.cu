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
//     magnitude < 2^15; over k <= 256 terms the sum stays below 2^23, so the
//     tensor core's FP32 accumulation is exact;
//   * C_ij = 2^{e_i + f_j} sum_{p+q <= P-1} 2^{-8(p+q+2)+2} (A_p B_q)_ij,
//     accumulated in FP64 (the 15 dropped pairs weigh at most 2^-62 each).
// The error is dominated by the 47-bit rounding, |dC_ij| <~ 2^-48 (2^{e_i}
// sum_k |B_kj| + 2^{f_j} sum_k |A_ik|), ~4e-15 relative to the row and column
// scales.  The slices are stored k-contiguous ([p][vector][k],
// k padded to a multiple of 32) for both operands, the layout the
// m16n8k16 row.col tensor instruction consumes.
#include <cuda_bf16.h>
#include <math.h>

#include "wpcd_internal.cuh"

namespace wpcd {

constexpr int kOzP = 6;    // slices per operand
constexpr int kOzKC = 32;  // k staged per step
constexpr int kOzLd = 40;  // padded shared row stride (bf16): conflict-free fragment loads
constexpr int kOzKMax = 256;  // k range whose FP32 sum of slice products is exact

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

__device__ __forceinline__ unsigned ld_u32(const __nv_bfloat16 *p) { return *reinterpret_cast<const unsigned *>(p); }

__device__ __forceinline__ void mma_bf16(float *c, unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                         unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// C[b] = A[b] B[b] from row slices of A and column slices of B.  64 x 64
// output tile per CTA, 4 warps of 32 x 32.
__global__ void __launch_bounds__(128) k_oz_gemm(int n, int Kp, const __nv_bfloat16 *A_s, const int *ea_all,
                                                 const __nv_bfloat16 *B_s, const int *eb_all, double *C_all)
{
    __shared__ __align__(16) __nv_bfloat16 As[64 * kOzLd];
    __shared__ __align__(16) __nv_bfloat16 Bs[64 * kOzLd];
    const int b = blockIdx.z;
    const int row0 = blockIdx.y * 64, col0 = blockIdx.x * 64;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g4 = lane >> 2, t = lane & 3;
    const int wr = (warp >> 1) * 32, wc = (warp & 1) * 32;
    const __nv_bfloat16 *Ab = A_s + (size_t)b * kOzP * n * Kp;
    const __nv_bfloat16 *Bb = B_s + (size_t)b * kOzP * n * Kp;

    double acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[i][j][u] = 0.0;

    // Digit pairs grouped by d = p + q (common weight 2^{-8(d+2)+2}).  Each
    // pair's FP32 sum over at most 256 k is an exact integer below 2^23; the
    // group adds them as int32 (at most 6 pairs x 2 k-chunks: below 2^27) and
    // reaches the FP64 accumulator once per group.
    for (int d = 0; d < kOzP; ++d) {
        int g[2][4][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int u = 0; u < 4; ++u) g[i][j][u] = 0;
        for (int p = 0; p <= d; ++p) {
            const int q = d - p;
            const __nv_bfloat16 *Ap = Ab + (size_t)p * n * Kp;
            const __nv_bfloat16 *Bq = Bb + (size_t)q * n * Kp;
            float c32[2][4][4];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int u = 0; u < 4; ++u) c32[i][j][u] = 0.f;
            for (int k0 = 0; k0 < Kp; k0 += kOzKC) {
                __syncthreads();
                // 64 rows x 32 k of each operand: 256 16-byte pieces each, 2 per thread
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int e = tid + u * 128;
                    const int r = e >> 2, kk = (e & 3) * 8;
                    uint4 va = make_uint4(0, 0, 0, 0), vb = make_uint4(0, 0, 0, 0);
                    if (row0 + r < n) va = *reinterpret_cast<const uint4 *>(Ap + (size_t)(row0 + r) * Kp + k0 + kk);
                    if (col0 + r < n) vb = *reinterpret_cast<const uint4 *>(Bq + (size_t)(col0 + r) * Kp + k0 + kk);
                    *reinterpret_cast<uint4 *>(&As[r * kOzLd + kk]) = va;
                    *reinterpret_cast<uint4 *>(&Bs[r * kOzLd + kk]) = vb;
                }
                __syncthreads();
#pragma unroll
                for (int ks = 0; ks < kOzKC; ks += 16) {
                    unsigned af[2][4], bf[4][2];
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const __nv_bfloat16 *base = &As[(wr + i * 16 + g4) * kOzLd + ks + 2 * t];
                        af[i][0] = ld_u32(base);
                        af[i][1] = ld_u32(base + 8 * kOzLd);
                        af[i][2] = ld_u32(base + 8);
                        af[i][3] = ld_u32(base + 8 * kOzLd + 8);
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const __nv_bfloat16 *base = &Bs[(wc + j * 8 + g4) * kOzLd + ks + 2 * t];
                        bf[j][0] = ld_u32(base);
                        bf[j][1] = ld_u32(base + 8);
                    }
#pragma unroll
                    for (int i = 0; i < 2; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            mma_bf16(c32[i][j], af[i][0], af[i][1], af[i][2], af[i][3], bf[j][0], bf[j][1]);
                }
                if (((k0 + kOzKC) % kOzKMax) == 0 || k0 + kOzKC >= Kp) {  // keep every FP32 sum exact
#pragma unroll
                    for (int i = 0; i < 2; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j)
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                g[i][j][u] += __float2int_rn(c32[i][j][u]);
                                c32[i][j][u] = 0.f;
                            }
                }
            }
        }
        const double scale = ldexp(1.0, -8 * (d + 2) + 2);  // digit weights 2^{-8(p+1)+1}
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[i][j][u] = fma((double)g[i][j][u], scale, acc[i][j][u]);
    }
    const int *ea = ea_all + (size_t)b * n, *eb = eb_all + (size_t)b * n;
    double *C = C_all + (size_t)b * n * n;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int r = row0 + wr + i * 16 + g4 + (u >= 2 ? 8 : 0);
                const int c = col0 + wc + j * 8 + 2 * t + (u & 1);
                if (r < n && c < n) C[(size_t)r * n + c] = ldexp(acc[i][j][u], ea[r] + eb[c]);
            }
}

// C = op(A) B for `items` n x n FP64 matrices (op(A) = A^T when ta), through
// the slices.  Scratch: sa, sb hold oz_slice_elems(n) bf16 per item; ea, eb n ints per item.
cudaError_t launch_oz_gemm(int n, int items, bool ta, const double *A, const double *B, double *C,
                           __nv_bfloat16 *sa, __nv_bfloat16 *sb, int *ea, int *eb, cudaStream_t st)
{
    const int Kp = oz_kpad(n);
    // rows of op(A): rows of A, or columns of A when transposed; columns of B
    const dim3 gcol((n + 127) / 128, items), grow((n + 7) / 8, items);
    const dim3 grows((Kp + 127) / 128, n, items), gtile((n + 31) / 32, (Kp + 31) / 32, items);
    if (ta) {
        k_oz_exp<true><<<gcol, 128, 0, st>>>(n, A, ea);
        k_oz_split_cols<<<gtile, dim3(32, 8), 0, st>>>(n, Kp, A, ea, sa);
    } else {
        k_oz_exp<false><<<grow, 256, 0, st>>>(n, A, ea);
        k_oz_split_rows<<<grows, 128, 0, st>>>(n, Kp, A, ea, sa);
    }
    k_oz_exp<true><<<gcol, 128, 0, st>>>(n, B, eb);
    k_oz_split_cols<<<gtile, dim3(32, 8), 0, st>>>(n, Kp, B, eb, sb);
    const int tiles = (n + 63) / 64;
    k_oz_gemm<<<dim3(tiles, tiles, items), 128, 0, st>>>(n, Kp, sa, ea, sb, eb, C);
    return cudaGetLastError();
}

}  // namespace wpcd
