// refine.cu -- FP64 refinement of approximate eigenpairs (mixed path).
//
// The FP32 eigensolve leaves eigenvectors X whose errors reach ~1e-4 inside
// the closely spaced low-energy part of the spectrum.  Each refinement
// iteration (Ogita & Aishima, "Iterative refinement for symmetric eigenvalue
// decomposition", 2018) computes in FP64
//     Y = H X,  S = X^T Y,  G = X^T X,  R = I - G,
//     lambda_i = S_ii / G_ii,
//     E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i)   if |lambda_j - lambda_i| > delta,
//     E_ij = R_ij / 2                                         otherwise (and on the diagonal),
//     delta = 2 (||S - diag(lambda)||_F + max|lambda| ||R||_F),
//     X <- X (I + E),
// which squares the eigenvector error.  The eigenvalues are the last
// iteration's FP64 Rayleigh quotients lambda_i = (X^T H X)_ii / (X^T X)_ii
// (quadratically accurate in the eigenvector error; the last update changes
// them below FP64 resolution).  The FP64 H comes from the FP32 solve,
// which forms it before rounding.  The four products are batched FP64
// GEMMs over every (sample, channel) item of one chunk of a size bucket; the
// working matrices of item b sit contiguously at b * n^2 in scratch buffers,
// and the final sort writes the eigenpairs into the eigen-buffer layout
// (channel offset + sample * n^2).
#include <cuda_bf16.h>
#include <math.h>

#include "wpcd_internal.cuh"

namespace wpcd {

// Batched C = op(A) B (n x n, row-major), op(A) = A^T when TA.  64 x 64 output
// tile per CTA, 16-deep k steps through shared memory, 4 x 4 outputs per thread.
constexpr int kBM = 64, kBK = 16;

template <bool TA>
__global__ void __launch_bounds__(256) k_bgemm64(int n, const double *A_all, const double *B_all, double *C_all)
{
    __shared__ double As[kBK][kBM];
    __shared__ double Bs[kBK][kBM];
    const size_t off = (size_t)blockIdx.z * n * n;
    const double *A = A_all + off, *B = B_all + off;
    double *C = C_all + off;
    const int row0 = blockIdx.y * kBM, col0 = blockIdx.x * kBM;
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < n; k0 += kBK) {
        // op(A) tile [rows row0.., k k0..] stored k-major; B tile [k, cols] stored k-major
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = tid + u * 256;  // 0..1023
            int kk, r;
            if (TA) {  // op(A)[r][k] = A[k][r]: read along r (coalesced)
                kk = e / kBM;
                r = e % kBM;
            } else {   // A[r][k]: read along k
                r = e / kBK;
                kk = e % kBK;
            }
            const int gr = row0 + r, gk = k0 + kk;
            double v = 0.0;
            if (gr < n && gk < n) v = TA ? A[(size_t)gk * n + gr] : A[(size_t)gr * n + gk];
            As[kk][r] = v;
            const int bk = e / kBM, bc = e % kBM;
            const int gbk = k0 + bk, gbc = col0 + bc;
            Bs[bk][bc] = (gbk < n && gbc < n) ? B[(size_t)gbk * n + gbc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            double a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gr = row0 + ty * 4 + i;
        if (gr >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gc = col0 + tx * 4 + j;
            if (gc < n) C[(size_t)gr * n + gc] = acc[i][j];
        }
    }
}

// One CTA per item: lambda, the threshold delta, and I + E written over G.
// Warp per row, lanes along the row.  Only what needs FP64 stays FP64: the
// Rayleigh quotients, lambda_j - lambda_i and the numerator S_ij + lambda_j R_ij
// (both cancel for close eigenvalues).  E_ij = numerator / (lambda_j - lambda_i)
// is formed in FP32 (relative error ~2^-22): an E of size |E| then carries an
// error ~|E| 2^-22, below 1e-15 once the second iteration's |E| ~ 1e-8.  The
// Frobenius norms of the threshold are FP32 sums.
__global__ void __launch_bounds__(256) k_oa_update(int n, const double *S_all, double *G_all, double *lam_all)
{
    extern __shared__ double lam[];  // n
    __shared__ double red[32];
    const int b = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const size_t off = (size_t)b * n * n;
    const double *S = S_all + off;
    double *G = G_all + off;
    double dsd = 0.0, drr = 0.0;  // diagonal terms in FP64
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double sii = S[(size_t)i * n + i], gii = G[(size_t)i * n + i];
        const double li = sii / gii;
        lam[i] = li;
        const double si = sii - li, ri = 1.0 - gii;
        dsd = fma(si, si, dsd);
        drr = fma(ri, ri, drr);
    }
    __syncthreads();
    float fsd = 0.0f, frr = 0.0f;
    for (int i = warp; i < n; i += nwarp) {
        const double *Si = S + (size_t)i * n, *Gi = G + (size_t)i * n;
        for (int j = lane; j < n; j += 32) {
            if (j == i) continue;
            const float s = f32_trunc(Si[j]), r = f32_trunc(Gi[j]);
            fsd = fmaf(s, s, fsd);
            frr = fmaf(r, r, frr);
        }
    }
    const double sd = cta_sum64(dsd + (double)fsd, red);
    const double rr = cta_sum64(drr + (double)frr, red);
    // ||H||_2 estimated by the largest |lambda| (Frobenius norms bound the other two)
    double lmax = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) lmax = fmax(lmax, fabs(lam[i]));
    for (int o = 16; o > 0; o >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    __syncthreads();
    if (lane == 0) red[warp] = lmax;
    __syncthreads();
    lmax = 0.0;
    for (int w = 0; w < nwarp; ++w) lmax = fmax(lmax, red[w]);
    const float delta = (float)(2.0 * (sqrt(sd) + lmax * sqrt(rr)));
    for (int i = warp; i < n; i += nwarp) {
        const double *Si = S + (size_t)i * n;
        double *Gi = G + (size_t)i * n;
        const double li = lam[i];
        for (int j = lane; j < n; j += 32) {
            const double g = Gi[j];
            if (j == i) {
                Gi[j] = 1.0 + 0.5 * (1.0 - g);
                continue;
            }
            const float dl = f32_trunc(lam[j] - li);
            float E;
            if (fabsf(dl) > delta) E = f32_trunc(fma(lam[j], -g, Si[j])) * __frcp_rn(dl);  // R_ij = -G_ij
            else E = -0.5f * f32_trunc(g);
            Gi[j] = f64_of(E);
        }
    }
    double *lo = lam_all + (size_t)b * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) lo[i] = lam[i];
}

// Sort the eigenvalues ascending and write them, with the columns of X
// permuted alike, into the eigen-buffer layout of their (sample, channel).
__global__ void __launch_bounds__(256) k_sort_eig(const ChanDev *chans, const int *work, int nw, int sample0, int n,
                                                  const double *lam_s, const double *X_s, double *eps_all,
                                                  double *X_all)
{
    extern __shared__ double sm[];
    double *lam = sm;                               // n
    int *rank = reinterpret_cast<int *>(lam + n);   // n
    const int b = blockIdx.x;
    const int wc = b % nw, smp = sample0 + b / nw;
    const ChanDev ch = chans[work[wc]];
    const double *Xs = X_s + (size_t)b * n * n;
    double *X = X_all + ch.c_off + (size_t)smp * n * n;
    double *eps = eps_all + ch.eps_off + (size_t)smp * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) lam[i] = lam_s[(size_t)b * n + i];
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double ei = lam[i];
        int r = 0;
        for (int j = 0; j < n; ++j) r += (lam[j] < ei) || (lam[j] == ei && j < i);
        rank[i] = r;
        eps[r] = ei;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int row = e / n, c = e - row * n;
        X[(size_t)row * n + rank[c]] = Xs[e];
    }
}

size_t sort_eig_smem(int n) { return (size_t)n * 8 + (size_t)n * 4; }

size_t refine_scratch_per_item(int n, int engine)
{
    size_t b = (size_t)5 * n * n * 8 + (size_t)n * 8;  // X, H, Y, W1, W2, lambda
    if (engine == 0) b += 5 * oz_slice_elems(n) * 2 + (size_t)5 * n * 4 + 512;  // 5 digit-slice sets
    return b;
}

// Refine the eigenpairs of `items` = n_samples * nw items of one bucket chunk.
// scratch: refine_scratch_per_item(n, engine) bytes per item, carved here.
// On entry Xs (the first n^2-double block of each item) holds the FP32-solve
// eigenvectors as FP64 and H (the second block) the FP64 Hamiltonian, both
// written by the FP32 solve.
// rot_s, rot_e (tensor engine only): the digit slices of the rows of the nw
// channels' basis matrices C0 when H and X are given in that basis (C0^T H C0
// and its eigenvectors X'); the refined vectors are then rotated back, X = C0 X',
// before the sort.
cudaError_t launch_refine(const ChanDev *chans, const int *work, int nw, int n_samples, int sample0, int n,
                          int n_terms, const double *coeffs, void *scratch, double *eps_all, double *X_all,
                          int iters, int engine, cudaStream_t st, int *err, const __nv_bfloat16 *rot_s,
                          const int *rot_e, int digits)
{
    if (digits < 4 || digits > kOzDigits) return cudaErrorInvalidValue;
    if (rot_s && engine != 0) return cudaErrorInvalidValue;
    (void)n_terms;
    (void)coeffs;
    if (iters < 0) return cudaErrorInvalidValue;
    const int items = n_samples * nw;
    const size_t nn = (size_t)items * n * n;
    double *Xs = static_cast<double *>(scratch);
    double *H = Xs + nn, *Y = H + nn, *W1 = Y + nn, *W2 = W1 + nn, *lam = W2 + nn;
    // digit slices start on a 256-byte boundary (16-byte vector loads)
    const uintptr_t s0 = (reinterpret_cast<uintptr_t>(lam + (size_t)items * n) + 255) & ~(uintptr_t)255;
    const size_t se = (size_t)items * oz_slice_elems(n);
    __nv_bfloat16 *sH = reinterpret_cast<__nv_bfloat16 *>(s0);
    __nv_bfloat16 *sXc = sH + se, *sYc = sXc + se, *sXr = sYc + se, *sEc = sXr + se;
    int *eH = reinterpret_cast<int *>(sEc + se);
    int *eXc = eH + (size_t)items * n, *eYc = eXc + (size_t)items * n, *eXr = eYc + (size_t)items * n;
    int *eEc = eXr + (size_t)items * n;
    const int tiles = (n + kBM - 1) / kBM;
    const dim3 gg(tiles, tiles, items);
    cudaError_t e = cudaSuccess;
#define CKR(x)                       \
    do {                             \
        if ((e = (x)) != cudaSuccess) \
            return e;                \
    } while (0)
    double *x = Xs, *xn = Y;
    if (engine == 0) CKR(launch_oz_split(n, items, false, H, sH, eH, st));  // rows of H, reused
    for (int it = 0; it < iters; ++it) {
        // digits per operand (6 by default, FP64-accurate products): errors of
        // S = X^T H X are divided by eigenvalue gaps (~1e-6 of ||H||) in E, so
        // the digit count sets the refined accuracy of every iteration
        const int dg = digits;
        if (engine == 0) {
            CKR(launch_oz_split(n, items, true, x, sXc, eXc, st));                   // columns of X
            CKR(launch_oz_gemm_slices(n, items, sH, eH, sXc, eXc, xn, st, dg, false, err));       // Y = H X
            CKR(launch_oz_split(n, items, true, xn, sYc, eYc, st));                  // columns of Y
            // S = X^T H X and G = X^T X are symmetric: upper tiles, mirrored
            CKR(launch_oz_gemm_slices(n, items, sXc, eXc, sYc, eYc, W1, st, dg, true, err));  // S = X^T Y
            CKR(launch_oz_gemm_slices(n, items, sXc, eXc, sXc, eXc, W2, st, dg, true, err));  // G = X^T X
        } else {
            k_bgemm64<false><<<gg, 256, 0, counted(st)>>>(n, H, x, xn);
            k_bgemm64<true><<<gg, 256, 0, counted(st)>>>(n, x, xn, W1);
            k_bgemm64<true><<<gg, 256, 0, counted(st)>>>(n, x, x, W2);
        }
        k_oa_update<<<items, 256, (size_t)n * 8, counted(st)>>>(n, W1, W2, lam);
        if (engine == 0) {
            CKR(launch_oz_split(n, items, false, x, sXr, eXr, st));              // rows of X
            CKR(launch_oz_split(n, items, true, W2, sEc, eEc, st));              // columns of I + E
            CKR(launch_oz_gemm_slices(n, items, sXr, eXr, sEc, eEc, xn, st, dg, false, err)); // X (I + E)
        } else {
            k_bgemm64<false><<<gg, 256, 0, counted(st)>>>(n, x, W2, xn);
        }
        double *t = x;
        x = xn;
        xn = t;
    }
    // lam holds the last iteration's Rayleigh quotients S_ii / G_ii of the vectors
    // entering it; its update moves each vector by |E| ~ 1e-8 and a Rayleigh
    // quotient by O(|E|^2 ||H||), below FP64 resolution, so no further H X is formed
    const double *xout = x;  // the refined vectors (Xs after an even number of iterations, else Y)
    if (rot_s) {
        // X = C0 X' (the same C0 for every sample of a channel: items run channel-fastest)
        CKR(launch_oz_split(n, items, true, x, sXc, eXc, st));
        CKR(launch_oz_gemm_slices(n, items, rot_s, rot_e, sXc, eXc, xn, st, digits, false, err, nw));
        xout = xn;
    }
#undef CKR
    k_sort_eig<<<items, 256, sort_eig_smem(n), counted(st)>>>(chans, work, nw, sample0, n, lam, xout, eps_all, X_all);
    return cudaGetLastError();
}

// Batched products through either engine (exposed for tests and callers).
cudaError_t launch_batched_dgemm(int n, int items, bool ta, const double *A, const double *B, double *C,
                                 void *scratch, int engine, cudaStream_t st, int *err)
{
    if (engine == 0) {
        __nv_bfloat16 *sa = static_cast<__nv_bfloat16 *>(scratch);
        __nv_bfloat16 *sb = sa + (size_t)items * oz_slice_elems(n);
        int *ea = reinterpret_cast<int *>(sb + (size_t)items * oz_slice_elems(n));
        return launch_oz_gemm(n, items, ta, A, B, C, sa, sb, ea, ea + (size_t)items * n, st, err);
    }
    const int tiles = (n + kBM - 1) / kBM;
    const dim3 gg(tiles, tiles, items);
    if (ta) k_bgemm64<true><<<gg, 256, 0, counted(st)>>>(n, A, B, C);
    else k_bgemm64<false><<<gg, 256, 0, counted(st)>>>(n, A, B, C);
    return cudaGetLastError();
}

size_t batched_dgemm_scratch(int n, int items) { return (size_t)items * (2 * oz_slice_elems(n) * 2 + 2 * n * 4) + 512; }

}  // namespace wpcd
