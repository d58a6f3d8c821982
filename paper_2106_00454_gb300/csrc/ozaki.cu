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
//     accumulated exactly in int64 and rounded once to FP64 (the 15 dropped
//     pairs weigh at most 2^-62 each).
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

// v 2^e as a double (round half away from zero), from the IEEE-754 layout with
// integer operations only; FP64 arithmetic only where the result leaves the
// normal range.
__device__ __forceinline__ double i64_times_pow2(long long v, int e)
{
    if (v == 0) return 0.0;
    unsigned long long m = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    int msb = 63 - __clzll((long long)m);
    unsigned long long frac;
    if (msb > 52) {
        int sh = msb - 52;
        m += 1ull << (sh - 1);  // m < 2^63: no overflow
        if (m >> (msb + 1)) {   // the rounding carried into a new leading bit
            ++msb;
            ++sh;
        }
        frac = m >> sh;
    } else {
        frac = m << (52 - msb);
    }
    const int be = msb + e + 1023;
    if (be < 1 || be > 2046) return ldexp((double)v, e);
    const unsigned long long bits =
        (v < 0 ? (1ull << 63) : 0ull) | ((unsigned long long)be << 52) | (frac & ((1ull << 52) - 1));
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// 16-byte global -> shared copy; src_bytes = 0 fills the 16 bytes with zeros.
__device__ __forceinline__ void cp_async16(unsigned dst, const void *src, int src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }

__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

constexpr int kOzStages = 3;                 // cp.async ring depth
constexpr int kOzStageElems = 2 * 64 * kOzLd;  // A and B tiles of one step (bf16)

// C[b] = A[b] B[b] from row slices of A and column slices of B, with the digit
// pairs p + q <= dmax (dmax = P - 1: every pair of weight >= 2^-40; a smaller
// dmax truncates the product to about 8 (dmax + 1) - 2 bits).  64 x 64
// output tile per CTA, 4 warps of 32 x 32.  The (digit pair, k-chunk) steps
// run as one sequence through a 3-stage cp.async ring, so the loads of step
// t + 2 overlap the tensor-core work of step t; fragments come from shared
// memory through ldmatrix.  sym: the product is known to be symmetric (X^T X,
// X^T H X); only tiles on and above the diagonal are formed, each written with
// its mirror.
__global__ void __launch_bounds__(128) k_oz_gemm(int n, int Kp, int dmax, bool sym, const __nv_bfloat16 *A_s,
                                                 const int *ea_all, const __nv_bfloat16 *B_s, const int *eb_all,
                                                 double *C_all)
{
    __shared__ __align__(128) __nv_bfloat16 ring[kOzStages * kOzStageElems];
    const int b = blockIdx.z;
    int tr = blockIdx.y, tc = blockIdx.x;
    if (sym) {  // a symmetric product: blockIdx.x enumerates the tiles tr <= tc only
        const int T = (n + 63) / 64;
        int e = blockIdx.x;
        tr = 0;
        while (e >= T - tr) {
            e -= T - tr;
            ++tr;
        }
        tc = tr + e;
    }
    const int row0 = tr * 64, col0 = tc * 64;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g4 = lane >> 2, t = lane & 3;
    const int wr = (warp >> 1) * 32, wc = (warp & 1) * 32;
    const __nv_bfloat16 *Ab = A_s + (size_t)b * kOzP * n * Kp;
    const __nv_bfloat16 *Bb = B_s + (size_t)b * kOzP * n * Kp;
    const int nk = Kp / kOzKC;                           // k-chunks per digit pair
    const int n_steps = nk * ((dmax + 1) * (dmax + 2) / 2);  // pairs p + q <= dmax (21 for dmax = P - 1)
    const unsigned ring_s = smem_u32(ring);

    // issue cursor: the (d, p, chunk) of the next step to load
    int id = 0, ip = 0, ik = 0;
    auto issue = [&](int stage) {
        const int q = id - ip;
        const __nv_bfloat16 *Ap = Ab + (size_t)ip * n * Kp;
        const __nv_bfloat16 *Bq = Bb + (size_t)q * n * Kp;
        const unsigned sA = ring_s + (unsigned)(stage * kOzStageElems) * 2u;
        const unsigned sB = sA + 64u * kOzLd * 2u;
#pragma unroll
        for (int u = 0; u < 2; ++u) {  // 64 rows x 32 k of each operand: 256 16-byte pieces, 2 per thread
            const int e = tid + u * 128;
            const int r = e >> 2, kk = (e & 3) * 8;
            const int ra = row0 + r < n ? row0 + r : n - 1, rb = col0 + r < n ? col0 + r : n - 1;
            cp_async16(sA + (unsigned)(r * kOzLd + kk) * 2u, Ap + (size_t)ra * Kp + ik * kOzKC + kk,
                       row0 + r < n ? 16 : 0);
            cp_async16(sB + (unsigned)(r * kOzLd + kk) * 2u, Bq + (size_t)rb * Kp + ik * kOzKC + kk,
                       col0 + r < n ? 16 : 0);
        }
        if (++ik == nk) {
            ik = 0;
            if (++ip > id) {
                ip = 0;
                ++id;
            }
        }
    };

    // v = sum over pairs of their sums times 2^{36-8d} (for d = 5 shifted down
    // by 4 bits instead): C_ij = v 2^{e_i + f_j - 50}, exact up to those 4 bits.
    long long acc[2][4][4];
    float c32[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                acc[i][j][u] = 0;
                c32[i][j][u] = 0.f;
            }

    // Digit pair (p, q) weighs 2^{-8(d+2)+2}, d = p + q.  Its FP32 sum over
    // at most 256 k is an exact integer of magnitude at most 256 * 129 * 128
    // < 2^23; it joins the int64 accumulator shifted by 36 - 8d (|v| < 2^62:
    // at most 6 pairs x 2 k-blocks of 2^22 per d), with no FP64 arithmetic.
    issue(0);
    cp_async_commit();
    if (n_steps > 1) issue(1);
    cp_async_commit();
    int cd = 0, cp = 0, ck = 0;  // compute cursor
    for (int st = 0; st < n_steps; ++st) {
        cp_async_wait1();  // step st has landed (only the newest group may be in flight)
        __syncthreads();   // ... for every thread, and step st - 1's stage is free again
        if (st + 2 < n_steps) issue((st + 2) % kOzStages);
        cp_async_commit();
        const unsigned sA = ring_s + (unsigned)((st % kOzStages) * kOzStageElems) * 2u;
        const unsigned sB = sA + 64u * kOzLd * 2u;
#pragma unroll
        // a warp tile wholly past the matrix edge has nothing to compute
        const bool live = row0 + wr < n && col0 + wc < n;
        for (int ks = 0; ks < kOzKC && live; ks += 16) {
            unsigned af[2][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {  // rows wr + 16 i + (lane & 15), k ks + 8 (lane >> 4)
                const int r = wr + i * 16 + (lane & 15), k = ks + 8 * (lane >> 4);
                ldsm_x4(sA + (unsigned)(r * kOzLd + k) * 2u, af[i][0], af[i][1], af[i][2], af[i][3]);
            }
#pragma unroll
            for (int jj = 0; jj < 2; ++jj) {  // columns wc + 16 jj + 8 (m >> 1) + (lane & 7), k ks + 8 (m & 1)
                const int m = lane >> 3;
                const int r = wc + jj * 16 + 8 * (m >> 1) + (lane & 7), k = ks + 8 * (m & 1);
                ldsm_x4(sB + (unsigned)(r * kOzLd + k) * 2u, bf[2 * jj][0], bf[2 * jj][1], bf[2 * jj + 1][0],
                        bf[2 * jj + 1][1]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    mma_bf16(c32[i][j], af[i][0], af[i][1], af[i][2], af[i][3], bf[j][0], bf[j][1]);
        }
        const int k_end = (ck + 1) * kOzKC;
        if ((k_end % kOzKMax) == 0 || ck + 1 == nk) {  // keep every FP32 sum exact
            const int sh = 36 - 8 * cd;                 // weight 2^{-8(d+2)+2} = 2^{sh-50}
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int v = __float2int_rn(c32[i][j][u]);
                        acc[i][j][u] += sh >= 0 ? ((long long)v << sh) : (long long)(v >> -sh);
                        c32[i][j][u] = 0.f;
                    }
        }
        if (++ck == nk) {
            ck = 0;
            if (++cp > cd) {
                cp = 0;
                ++cd;
            }
        }
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
                if (r < n && c < n) {
                    const double v = i64_times_pow2(acc[i][j][u], ea[r] + eb[c] - 50);
                    C[(size_t)r * n + c] = v;
                    if (sym && tr != tc) C[(size_t)c * n + r] = v;  // the mirrored tile
                }
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
                                  const int *eb, double *C, cudaStream_t st, int digits, bool sym)
{
    if (digits < 1 || digits > kOzP) return cudaErrorInvalidValue;
    const int tiles = (n + 63) / 64;
    if (sym)
        k_oz_gemm<<<dim3(tiles * (tiles + 1) / 2, 1, items), 128, 0, st>>>(n, oz_kpad(n), digits - 1, true, sa, ea, sb,
                                                                            eb, C);
    else
        k_oz_gemm<<<dim3(tiles, tiles, items), 128, 0, st>>>(n, oz_kpad(n), digits - 1, false, sa, ea, sb, eb, C);
    return cudaGetLastError();
}

cudaError_t launch_oz_gemm(int n, int items, bool ta, const double *A, const double *B, double *C,
                           __nv_bfloat16 *sa, __nv_bfloat16 *sb, int *ea, int *eb, cudaStream_t st)
{
    cudaError_t e;
    // rows of op(A): rows of A, or columns of A when transposed; columns of B
    if ((e = launch_oz_split(n, items, ta, A, sa, ea, st))) return e;
    if ((e = launch_oz_split(n, items, true, B, sb, eb, st))) return e;
    return launch_oz_gemm_slices(n, items, sa, ea, sb, eb, C, st);
}

}  // namespace wpcd
