// eig_mixed.cu -- (a2, a3) reduced-precision eigensolve with FP64 refinement.
//
// H = diag(H0) + V0 + sum_a c_a V_a is formed in FP64 and rounded to FP32 in
// shared memory; the parallel cyclic Jacobi method of the FP64 kernel then
// runs in FP32 (GB300 issues FP32 at 58x its FP64 rate).  A pair is rotated
// only while |a_pq| > 2^-23 sqrt|a_pp a_qq|, the relative test that lets
// Jacobi resolve small eigenvalues of a graded matrix to their own relative
// accuracy; the sweeps stop after a sweep that rotates nothing.  The
// eigenvectors leave as FP64 (exact copies of the FP32 values), unsorted, in a
// contiguous scratch layout [item][n][n], for the FP64 refinement that follows.
#include <math.h>

#include "wpcd_internal.cuh"

namespace wpcd {

constexpr int kMixMaxThreads = 512;  // launch bound; the launch picks 64..512
constexpr int kMixMaxSweeps = 40;
constexpr size_t kMixSmemCap = 200 * 1024;
constexpr float kRelTol = 1.1920929e-7f;  // 2^-23

__host__ __device__ inline int mpad(int n) { return (n + 1) & ~1; }
__host__ __device__ inline size_t mpacked(int n) { return (size_t)n * (n + 1) / 2; }

// Index pairs (P, P2), P < P2, of the rotation slots whose 2 x 2 blocks of A
// one round updates: h (h - 1) / 2 of them, 8 bits each (h <= 256, which
// every A that fits in shared memory satisfies).
__host__ __device__ inline int mquads(int n)
{
    const int h = mpad(n) / 2;
    return h * (h - 1) / 2;
}

// A float packed (>= 10 n floats) | cos, sin, a_pp', a_qq' float [h] | p, q int [h] |
// reduction double [64] | rank int [n, even] | flags int [2] | slot pairs ushort [quads, even] |
// C float [n*n]
__host__ __device__ inline size_t mix_smem(int n, bool c_in_smem)
{
    const int h = mpad(n) / 2;
    size_t a = mpacked(n);
    if (a < (size_t)10 * n) a = (size_t)10 * n;
    a = (a + 1) & ~(size_t)1;  // keep the next region 8-byte aligned
    size_t b = a * 4 + (size_t)4 * h * 4 + (size_t)2 * h * 4;
    b = (b + 7) & ~(size_t)7;
    b += 64 * 8 + (size_t)mpad(n) * 4 + 2 * 4;
    b += (size_t)((mquads(n) + 1) & ~1) * 2;
    if (c_in_smem) b += (size_t)n * n * 4;
    return b;
}

size_t jacobi_mixed_smem_bytes(int n, bool c_in_smem) { return mix_smem(n, c_in_smem); }

template <bool C_SMEM>
__global__ void __launch_bounds__(kMixMaxThreads) k_jacobi_mixed(const ChanDev *chans, const int *work_ch, int n_work_ch,
                                                               int sample0, int n_terms, const double *coeffs,
                                                               double *lam_s, double *X_s, float *Cf_s,
                                                               double *H_s, int *status_all, int n_ch_total, int *err)
{
    const int wc = blockIdx.x % n_work_ch;
    const int smp = sample0 + blockIdx.x / n_work_ch;
    const int cidx = work_ch[wc];
    const ChanDev ch = chans[cidx];
    const int n = ch.n, N = ch.N, npad = mpad(n), h = npad / 2;
    const int tid = threadIdx.x, nt = blockDim.x;
    if ((size_t)dyn_smem_bytes() < mix_smem(n, C_SMEM)) {
        if (tid == 0) {
            status_all[(size_t)smp * n_ch_total + cidx] = -1;
            record_error(err, kDevBadSize);
        }
        return;
    }
    extern __shared__ double smem_d[];
    unsigned char *sb = reinterpret_cast<unsigned char *>(smem_d);
    size_t alen = mpacked(n);
    if (alen < (size_t)10 * n) alen = (size_t)10 * n;
    alen = (alen + 1) & ~(size_t)1;
    float *A = reinterpret_cast<float *>(sb);
    float *rc = A + alen, *rs = rc + h, *dpp = rs + h, *dqq = dpp + h;
    int *pp_ = reinterpret_cast<int *>(dqq + h), *qq_ = pp_ + h;
    size_t off = (alen + 4 * (size_t)h) * 4 + (size_t)2 * h * 4;
    off = (off + 7) & ~(size_t)7;
    double *red = reinterpret_cast<double *>(sb + off);
    int *rank = reinterpret_cast<int *>(red + 64);
    int *flags = rank + npad;
    unsigned short *quad = reinterpret_cast<unsigned short *>(flags + 2);
    const int nq = mquads(n);
    float *Cs = C_SMEM ? reinterpret_cast<float *>(quad + ((nq + 1) & ~1)) : nullptr;
    float *Cg = Cf_s + (size_t)blockIdx.x * n * n;
    float *C = C_SMEM ? Cs : Cg;
    const double *cf = coeffs ? coeffs + (size_t)smp * (n_terms - 1) : nullptr;

    // ---- H in FP64, rounded to FP32; the FP64 H also goes to H_s for the refinement
    double *Hg = H_s ? H_s + (size_t)blockIdx.x * n * n : nullptr;
    for (int e = tid; e < n * n; e += nt) {
        int i = e / n, j = e - i * n;
        if (i > j) continue;
        double v = ch.V[e];
        for (int a = 1; a < n_terms; ++a) v = fma(cf[a - 1], ch.V[(size_t)a * n * n + e], v);
        if (i == j) v += ch.h0[i % N];
        A[pk(i, j)] = (float)v;
        if (Hg) {
            Hg[e] = v;
            Hg[(size_t)j * n + i] = v;
        }
    }
    for (int e = tid; e < n * n; e += nt) {
        int i = e / n, j = e - i * n;
        C[(size_t)i * n + j] = (i == j) ? 1.0f : 0.0f;
    }
    for (int e = tid; e < h * h; e += nt) {  // slot pairs in row order of P
        const int P = e / h, P2 = e - P * h;
        if (P < P2) quad[P * h - P * (P + 1) / 2 + (P2 - P - 1)] = (unsigned short)((P << 8) | P2);
    }
    __syncthreads();

    int sweeps = 0;
    bool converged = false;
    while (sweeps < kMixMaxSweeps) {
        if (tid == 0) flags[0] = 0;
        __syncthreads();
        ++sweeps;
        for (int r = 0; r < npad - 1; ++r) {
            for (int k = tid; k < h; k += nt) {
                int p, q;
                jac_pair_of(r, k, npad, p, q);
                pp_[k] = p;
                qq_[k] = q;
                float c = 1.0f, s = 0.0f, app = 0.0f, aqq = 0.0f;
                if (q < n) {
                    app = A[pk(p, p)];
                    aqq = A[pk(q, q)];
                    const float apq = A[pk(p, q)];
                    if (fabsf(apq) > kRelTol * sqrtf(fabsf(app) * fabsf(aqq))) {
                        const float tau = (aqq - app) / (2.0f * apq);
                        float t;
                        if (fabsf(tau) > 1e18f) t = 0.5f / tau;
                        else t = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
                        c = 1.0f / sqrtf(1.0f + t * t);
                        s = t * c;
                        app -= t * apq;
                        aqq += t * apq;
                        flags[0] = 1;
                    }
                }
                rc[k] = c;
                rs[k] = s;
                dpp[k] = app;
                dqq[k] = aqq;
            }
            __syncthreads();
            for (int e = tid; e < nq; e += nt) {
                const unsigned pr = quad[e];
                const int P = pr >> 8, P2 = pr & 0xFF;
                const int p = pp_[P], q = qq_[P], p2 = pp_[P2], q2 = qq_[P2];
                const float c = rc[P], s = rs[P], c2 = rc[P2], s2 = rs[P2];
                if (s == 0.0f && s2 == 0.0f) continue;  // both rotations are the identity
                const bool qv = q < n, q2v = q2 < n;
                const float b00 = A[pk(p, p2)];
                const float b01 = q2v ? A[pk(p, q2)] : 0.0f;
                const float b10 = qv ? A[pk(q, p2)] : 0.0f;
                const float b11 = (qv && q2v) ? A[pk(q, q2)] : 0.0f;
                const float x00 = c2 * b00 - s2 * b01, x01 = s2 * b00 + c2 * b01;
                const float x10 = c2 * b10 - s2 * b11, x11 = s2 * b10 + c2 * b11;
                A[pk(p, p2)] = c * x00 - s * x10;
                if (q2v) A[pk(p, q2)] = c * x01 - s * x11;
                if (qv) A[pk(q, p2)] = s * x00 + c * x10;
                if (qv && q2v) A[pk(q, q2)] = s * x01 + c * x11;
            }
            for (int k = tid; k < h; k += nt) {
                const int p = pp_[k], q = qq_[k];
                if (q < n && rs[k] != 0.0f) {
                    A[pk(p, p)] = dpp[k];
                    A[pk(q, q)] = dqq[k];
                    A[pk(p, q)] = 0.0f;
                }
            }
            // C is kept column-major (column s contiguous): one warp per rotation,
            // its lanes walking consecutive rows of the two columns; a warp
            // skips an identity rotation as a whole
            for (int k = tid >> 5; k < h; k += nt >> 5) {
                const int p = pp_[k], q = qq_[k];
                const float s = rs[k];
                if (q >= n || s == 0.0f) continue;
                const float c = rc[k];
                float *Cp = C + (size_t)p * n, *Cq = C + (size_t)q * n;
                for (int row = tid & 31; row < n; row += 32) {
                    const float cp = Cp[row], cq = Cq[row];
                    Cp[row] = c * cp - s * cq;
                    Cq[row] = s * cp + c * cq;
                }
            }
            __syncthreads();
        }
        if (flags[0] == 0) {
            converged = true;
            break;
        }
        __syncthreads();
    }

    // ---- FP32 eigenpairs out, as FP64, unsorted
    double *X = X_s + (size_t)blockIdx.x * n * n;  // row-major out of the column-major C
    for (int e = tid; e < n * n; e += nt) {
        const int col = e / n, row = e - col * n;
        X[(size_t)row * n + col] = (double)C[e];
    }
    for (int i = tid; i < n; i += nt) lam_s[(size_t)blockIdx.x * n + i] = (double)A[pk(i, i)];
    if (tid == 0) {
        status_all[(size_t)smp * n_ch_total + cidx] = converged ? sweeps : -1;
        if (!converged) record_error(err, kDevNoConverge);
    }
}

cudaError_t launch_jacobi_mixed(const ChanDev *chans_dev, const int *work_ch_dev, int n_work_ch, int n_samples,
                                int sample0, int n_terms, const double *coeffs, int n, double *lam_s, double *X_s,
                                float *Cf_s, double *H_s, int *status_all, int n_ch_total, int *err, cudaStream_t st,
                                int threads)
{
    if (threads < 32 || threads > kMixMaxThreads || (threads & 31)) return cudaErrorInvalidValue;
    const bool cs = mix_smem(n, true) <= kMixSmemCap;
    const size_t smem = mix_smem(n, cs);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    dim3 grid((unsigned)(n_samples * n_work_ch));
    if (cs) {
        cudaFuncSetAttribute(k_jacobi_mixed<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_jacobi_mixed<true><<<grid, threads, smem, st>>>(chans_dev, work_ch_dev, n_work_ch, sample0, n_terms,
                                                              coeffs, lam_s, X_s, Cf_s, H_s, status_all, n_ch_total, err);
    } else {
        cudaFuncSetAttribute(k_jacobi_mixed<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_jacobi_mixed<false><<<grid, threads, smem, st>>>(chans_dev, work_ch_dev, n_work_ch, sample0, n_terms,
                                                               coeffs, lam_s, X_s, Cf_s, H_s, status_all, n_ch_total, err);
    }
    return cudaGetLastError();
}

bool jacobi_mixed_c_in_smem(int n) { return mix_smem(n, true) <= kMixSmemCap; }

int jacobi_mixed_occupancy(int n, int threads)
{
    const bool cs = mix_smem(n, true) <= kMixSmemCap;
    const size_t smem = mix_smem(n, cs);
    int blocks = 0;
    if (cs) {
        cudaFuncSetAttribute(k_jacobi_mixed<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_jacobi_mixed<true>, threads, smem);
    } else {
        cudaFuncSetAttribute(k_jacobi_mixed<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_jacobi_mixed<false>, threads, smem);
    }
    return blocks;
}

}  // namespace wpcd
