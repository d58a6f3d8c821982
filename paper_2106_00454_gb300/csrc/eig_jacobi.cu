// eig_jacobi.cu -- (a2) parameter sum + H assembly and (a3) symmetric
// eigendecomposition H = C D C^T (Sec. 3.2 step 2), FP64.
//
// One CTA per (sample, channel).  H = diag(H0) + V0 + sum_a c_a V_a is formed
// directly in shared memory (packed upper triangle), then diagonalised by the
// parallel cyclic two-sided Jacobi method (the method the paper's GPU code ran
// through a batched library call, Sec. 4.2.2 and App. C): each round applies
// n/2 disjoint rotations chosen by a round-robin tournament, so that every pair
// (p, q) is visited once per sweep.  A round is two phases:
//   1. every pair computes its rotation from (a_pp, a_qq, a_pq);
//   2. every 2x2 block (P, P') of A is replaced by J_P^T B J_P', the diagonal
//      blocks by (a_pp - t a_pq, a_qq + t a_pq) with a_pq = 0, and the columns
//      p, q of C are rotated.
// Sweeps stop when off(A) <= 1e-15 ||H||_F or after max_sweeps (status -1).
// Eigenvalues leave sorted ascending with the columns of C permuted alike.
#include <math.h>

#include "wpcd_internal.cuh"

namespace wpcd {

constexpr int kJacMaxThreads = 512;  // launch bound; the launch picks 64..512
constexpr int kMaxSweeps = 40;
constexpr size_t kSmemCap = 200 * 1024;

__host__ __device__ inline int npad_of(int n) { return (n + 1) & ~1; }
__host__ __device__ inline size_t packed_len(int n) { return (size_t)n * (n + 1) / 2; }

// Rotation-slot pairs (P, P2), P < P2, whose 2 x 2 blocks of A one round
// updates, 8 bits each (h <= 256 for every A that fits in shared memory).
__host__ __device__ inline int slot_pairs(int n)
{
    const int h = npad_of(n) / 2;
    return h * (h - 1) / 2;
}

// A (packed) | cos, sin, new a_pp, new a_qq [h each] | p, q [h ints each] | reduction [64] | rank [n, even] |
// C [n*n] | slot pairs ushort [even count]
__host__ __device__ inline size_t jacobi_smem_bytes_dev(int n, bool c_in_smem)
{
    int h = npad_of(n) / 2;
    size_t b = packed_len(n) * 8 + (size_t)4 * h * 8 + (size_t)2 * h * 4 + 64 * 8 + (size_t)((n + 1) & ~1) * 4;
    if (c_in_smem) b += (size_t)n * n * 8;
    b += (size_t)((slot_pairs(n) + 1) & ~1) * 2;
    return b;
}

size_t jacobi_smem_bytes(int n, bool c_in_smem) { return jacobi_smem_bytes_dev(n, c_in_smem); }

bool jacobi_c_in_smem(int n) { return jacobi_smem_bytes(n, true) <= kSmemCap; }

__device__ __forceinline__ void pair_of(int r, int k, int npad, int &p, int &q)
{
    const int M = npad - 1;
    int a, b;
    if (k == 0) {
        a = 0;
        b = 1 + (r % M);
    } else {
        a = 1 + (r + k) % M;
        b = 1 + (r - k + M) % M;
    }
    p = a < b ? a : b;
    q = a < b ? b : a;
}

__device__ __forceinline__ double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

template <bool C_SMEM>
__global__ void __launch_bounds__(kJacMaxThreads) k_jacobi_f64(const ChanDev *chans, const int *work_ch, int n_work_ch,
                                                             int sample0, int n_terms, const double *coeffs,
                                                             double *eps_all, double *C_all, int *status_all,
                                                             int n_ch_total, int *err)
{
    const int wc = blockIdx.x % n_work_ch;
    const int smp = sample0 + blockIdx.x / n_work_ch;
    const int cidx = work_ch[wc];
    const ChanDev ch = chans[cidx];
    const int n = ch.n, N = ch.N, npad = npad_of(n), h = npad / 2;
    const int tid = threadIdx.x, nt = blockDim.x;
    if ((size_t)dyn_smem_bytes() < jacobi_smem_bytes_dev(n, C_SMEM)) {  // launch/layout mismatch
        if (tid == 0) {
            status_all[(size_t)smp * n_ch_total + cidx] = -1;
            record_error(err, kDevBadSize);
        }
        return;
    }

    extern __shared__ double smem[];
    double *A = smem;                                 // packed upper, n(n+1)/2
    double *rc = A + packed_len(n);                   // cos [h]
    double *rs = rc + h;                              // sin [h]
    double *dpp = rs + h;                             // new a_pp [h]
    double *dqq = dpp + h;                            // new a_qq [h]
    int *pp_ = reinterpret_cast<int *>(dqq + h);      // p [h]
    int *qq_ = pp_ + h;                               // q [h]
    double *red = reinterpret_cast<double *>(pp_ + 2 * h);  // 64 doubles (8-byte aligned: 2h ints)
    int *rank = reinterpret_cast<int *>(red + 64);    // [n]
    double *Cs = nullptr;
    if (C_SMEM) Cs = reinterpret_cast<double *>(rank + ((n + 1) & ~1));
    unsigned short *quad = C_SMEM ? reinterpret_cast<unsigned short *>(Cs + (size_t)n * n)
                                  : reinterpret_cast<unsigned short *>(rank + ((n + 1) & ~1));
    const int nq = slot_pairs(n);

    double *Cg = C_all + ch.c_off + (size_t)smp * n * n;
    double *C = C_SMEM ? Cs : Cg;
    const double *cf = coeffs ? coeffs + (size_t)smp * (n_terms - 1) : nullptr;

    // ---- (a2) H = diag(H0) + V0 + sum_a c_a V_a, written into the packed upper triangle
    double fro2 = 0.0;
    for (int e = tid; e < n * n; e += nt) {
        int i = e / n, j = e - i * n;
        if (i > j) continue;
        double v = ch.V[e];
        for (int a = 1; a < n_terms; ++a) v = fma(cf[a - 1], ch.V[(size_t)a * n * n + e], v);
        if (i == j) v += ch.h0[i % N];
        A[pk(i, j)] = v;
        fro2 += (i == j ? 1.0 : 2.0) * v * v;
    }
    for (int e = tid; e < n * n; e += nt) {
        int i = e / n, j = e - i * n;
        C[(size_t)i * n + j] = (i == j) ? 1.0 : 0.0;
    }
    for (int e = tid; e < h * h; e += nt) {  // slot pairs in row order of P
        const int P = e / h, P2 = e - P * h;
        if (P < P2) quad[P * h - P * (P + 1) / 2 + (P2 - P - 1)] = (unsigned short)((P << 8) | P2);
    }
    fro2 = block_sum(fro2, red);
    const double tol2 = 1e-30 * fro2;  // (1e-15 ||H||_F)^2

    int sweeps = 0;
    bool converged = false;
    for (;;) {
        double off2 = 0.0;
        for (int e = tid; e < (int)packed_len(n); e += nt) {
            // column-major packed: recover (i, j) with i < j
            int j = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
            while ((j + 1) * (j + 2) / 2 <= e) ++j;
            while (j * (j + 1) / 2 > e) --j;
            int i = e - j * (j + 1) / 2;
            if (i != j) off2 += 2.0 * A[e] * A[e];
        }
        off2 = block_sum(off2, red);
        if (off2 <= tol2) { converged = true; break; }
        if (sweeps >= kMaxSweeps) break;
        ++sweeps;
        for (int r = 0; r < npad - 1; ++r) {
            // phase 1: rotations of this round
            for (int k = tid; k < h; k += nt) {
                int p, q;
                pair_of(r, k, npad, p, q);
                pp_[k] = p;
                qq_[k] = q;
                double c = 1.0, s = 0.0, app = 0.0, aqq = 0.0;
                if (q < n) {
                    app = A[pk(p, p)];
                    aqq = A[pk(q, q)];
                    double apq = A[pk(p, q)];
                    if (apq != 0.0) {
                        double tau = (aqq - app) / (2.0 * apq);
                        double t;
                        if (fabs(tau) > 1e150) t = 0.5 / tau;
                        else t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                        app -= t * apq;
                        aqq += t * apq;
                    }
                }
                rc[k] = c;
                rs[k] = s;
                dpp[k] = app;
                dqq[k] = aqq;
            }
            __syncthreads();
            // phase 2a: off-diagonal 2x2 blocks (P < P') -> J_P^T B J_P'
            for (int e = tid; e < nq; e += nt) {
                const unsigned pr = quad[e];
                const int P = pr >> 8, P2 = pr & 0xFF;
                const int p = pp_[P], q = qq_[P], p2 = pp_[P2], q2 = qq_[P2];
                const double c = rc[P], s = rs[P], c2 = rc[P2], s2 = rs[P2];
                if (s == 0.0 && s2 == 0.0) continue;  // both rotations are the identity
                const bool qv = q < n, q2v = q2 < n;
                double b00 = A[pk(p, p2)];
                double b01 = q2v ? A[pk(p, q2)] : 0.0;
                double b10 = qv ? A[pk(q, p2)] : 0.0;
                double b11 = (qv && q2v) ? A[pk(q, q2)] : 0.0;
                // B J' (columns p2, q2)
                double x00 = c2 * b00 - s2 * b01, x01 = s2 * b00 + c2 * b01;
                double x10 = c2 * b10 - s2 * b11, x11 = s2 * b10 + c2 * b11;
                // J^T (rows p, q)
                A[pk(p, p2)] = c * x00 - s * x10;
                if (q2v) A[pk(p, q2)] = c * x01 - s * x11;
                if (qv) A[pk(q, p2)] = s * x00 + c * x10;
                if (qv && q2v) A[pk(q, q2)] = s * x01 + c * x11;
            }
            // phase 2b: diagonal blocks
            for (int k = tid; k < h; k += nt) {
                int p = pp_[k], q = qq_[k];
                if (q < n) {
                    A[pk(p, p)] = dpp[k];
                    A[pk(q, q)] = dqq[k];
                    A[pk(p, q)] = 0.0;
                }
            }
            // phase 2c: columns p, q of C
            // one warp per rotation, its lanes walking the rows; identity rotations
            // are skipped by the whole warp
            for (int k = tid >> 5; k < h; k += nt >> 5) {
                const int p = pp_[k], q = qq_[k];
                const double s = rs[k];
                if (q >= n || s == 0.0) continue;
                const double c = rc[k];
                for (int row = tid & 31; row < n; row += 32) {
                    // in shared memory C is column-major (conflict-free row walks);
                    // in global memory it stays row-major for the in-place final permutation
                    const size_t ip = C_SMEM ? (size_t)p * n + row : (size_t)row * n + p;
                    const size_t iq = C_SMEM ? (size_t)q * n + row : (size_t)row * n + q;
                    const double cp = C[ip], cq = C[iq];
                    C[ip] = c * cp - s * cq;
                    C[iq] = s * cp + c * cq;
                }
            }
            __syncthreads();
        }
    }

    // ---- eigenvalues ascending (rank sort, ties by index) and permuted eigenvectors
    double *eps = eps_all + ch.eps_off + (size_t)smp * n;
    for (int i = tid; i < n; i += nt) {
        double ei = A[pk(i, i)];
        int r = 0;
        for (int j = 0; j < n; ++j) {
            double ej = A[pk(j, j)];
            r += (ej < ei) || (ej == ei && j < i);
        }
        rank[i] = r;
        eps[r] = ei;
    }
    __syncthreads();
    if (C_SMEM) {
        for (int e = tid; e < n * n; e += nt) {
            int row = e / n, col = e - row * n;
            Cg[(size_t)row * n + rank[col]] = Cs[(size_t)col * n + row];
        }
    } else {
        // permute in place row by row through the (now free) A storage
        const int nw = nt >> 5, w = tid >> 5, lane = tid & 31;
        double *buf = A + (size_t)w * n;
        for (int row = w; row < n; row += nw) {
            for (int col = lane; col < n; col += 32) buf[col] = Cg[(size_t)row * n + col];
            __syncwarp();
            for (int col = lane; col < n; col += 32) Cg[(size_t)row * n + rank[col]] = buf[col];
            __syncwarp();
        }
    }
    if (tid == 0) {
        status_all[(size_t)smp * n_ch_total + cidx] = converged ? sweeps : -1;
        if (!converged) record_error(err, kDevNoConverge);
    }
}

cudaError_t launch_jacobi_f64(const ChanDev *chans_dev, const int *work_ch_dev, int n_work_ch, int n_samples,
                              int sample0, int n_terms, const double *coeffs, int n, double *eps_all, double *C_all,
                              int *status_all, int n_ch_total, int *err, cudaStream_t st, int threads)
{
    if (threads < 32 || threads > kJacMaxThreads || (threads & 31)) return cudaErrorInvalidValue;
    bool cs = jacobi_c_in_smem(n);
    size_t smem = jacobi_smem_bytes(n, cs);
    if (!cs && (size_t)(threads / 32) * n > packed_len(n)) return cudaErrorInvalidValue;  // row buffers fit in A
    dim3 grid((unsigned)(n_samples * n_work_ch));
    if (cs) {
        raise_smem_limit((const void *)k_jacobi_f64<true>, smem);
        k_jacobi_f64<true><<<grid, threads, smem, counted(st)>>>(chans_dev, work_ch_dev, n_work_ch, sample0, n_terms,
                                                            coeffs, eps_all, C_all, status_all, n_ch_total, err);
    } else {
        raise_smem_limit((const void *)k_jacobi_f64<false>, smem);
        k_jacobi_f64<false><<<grid, threads, smem, counted(st)>>>(chans_dev, work_ch_dev, n_work_ch, sample0, n_terms,
                                                             coeffs, eps_all, C_all, status_all, n_ch_total, err);
    }
    return cudaGetLastError();
}

int jacobi_f64_occupancy(int n, int threads)
{
    const bool cs = jacobi_c_in_smem(n);
    const size_t smem = jacobi_smem_bytes(n, cs);
    int blocks = 0;
    if (cs) {
        raise_smem_limit((const void *)k_jacobi_f64<true>, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_jacobi_f64<true>, threads, smem);
    } else {
        raise_smem_limit((const void *)k_jacobi_f64<false>, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_jacobi_f64<false>, threads, smem);
    }
    return blocks;
}

}  // namespace wpcd
