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
// The eigenvectors C stay in shared memory while A, the tables and C fit in this
// many bytes (n <= 149), else they live in global memory (L2): from n = 150 on,
// the smaller CTAs without C run more solves per SM than their L2 round trips
// cost (measured at n = 150: 11.3 us per solve with C in shared memory and one
// 1024-thread CTA per SM, 8.2 us with C in L2 and 256-thread CTAs).
constexpr size_t kMixSmemCap = 150 * 1024;
constexpr float kRelTol = 1.1920929e-7f;  // 2^-23
// Threshold Jacobi (Rutishauser) on large matrices: in the first sweeps a pair
// rotates only if |a_pq| also exceeds kMixThreshFrac * off(A) / n, off(A) the
// Frobenius norm of the strict upper triangle at the sweep's start.  Measured on
// the 200 x 200 coupled blocks: the same number of sweeps with a third fewer
// rotations; on smaller matrices it costs extra sweeps, so it is kept to
// n >= kMixThreshN (where the eigenvector columns also live in global memory).
constexpr int kMixThreshN = 160;
constexpr int kMixThreshSweeps = 2;
constexpr float kMixThreshFrac = 0.1f;

__host__ __device__ inline int mpad(int n) { return (n + 1) & ~1; }
__host__ __device__ inline int mldc(int n) { return (n + 3) & ~3; }  // column stride of C: float4 rows

// A is stored as its upper triangle, column by column, with column y (rows
// 0..y) starting at mcol(y) == y (mod 32): element (x, y), x <= y, then lies in
// shared-memory bank (x + y) mod 32, whichever index is the larger.  A block
// update reads, across a warp, the elements of one slot's index with the
// indices of consecutive tournament slots, which run over consecutive values
// (r + k + 1 upwards, r - k + 1 downwards), so the 32 lanes of one access fall
// in 32 different banks, apart from a row change or a wrap of the tournament
// inside the warp.  (Columns packed back to back at y (y + 1) / 2 put two or
// more lanes in one bank on about half of those accesses.)  The padding is
// (-y) mod 32 floats after column y: 15.5 floats a column on average.
__host__ __device__ inline int mcol(int y)
{
    const int a = y >> 5, b = y & 31;
    return y * (y + 1) / 2 + 496 * a + (b ? (b - 1) * (64 - b) / 2 : 0);
}

// Index pairs (P, P2), P < P2, of the rotation slots whose 2 x 2 blocks of A
// one round updates: h (h - 1) / 2 of them in row order of P, 8 bits each
// (h <= 256, which every A that fits in shared memory satisfies).
__host__ __device__ inline int mquads(int n)
{
    const int h = mpad(n) / 2;
    return h * (h - 1) / 2;
}

__host__ __device__ inline size_t mix_a_floats(int n)
{
    const int np = mpad(n);  // the odd-n phantom row and column are kept (as zeros)
    size_t a = (size_t)mcol(np - 1) + np;
    if (a < (size_t)10 * n) a = (size_t)10 * n;
    return (a + 3) & ~(size_t)3;  // the slot records after it are 16-byte aligned
}

// A float [mix_a_floats] | slot records uint4 [h] {c, s', a | b << 16, mcol(a) | mcol(b) << 16} |
// a_aa', a_bb' float [h] each | flags int [8] | rank of each slot among the round's rotating
// slots int [h] | rotating slots ushort [h, even] | slot pairs ushort [quads, even] | (16-byte aligned)
// C float [n][ldc] (column-major) when it is kept in shared memory
__host__ __device__ inline size_t mix_smem(int n, bool c_in_smem)
{
    const int h = mpad(n) / 2;
    size_t b = mix_a_floats(n) * 4 + (size_t)h * (16 + 8) + 8 * 4 + (size_t)h * 4 + (size_t)((h + 1) & ~1) * 2;
    b += (size_t)((mquads(n) + 1) & ~1) * 2;
    b = (b + 15) & ~(size_t)15;
    if (c_in_smem) b += (size_t)n * mldc(n) * 4;
    return b;
}

size_t jacobi_mixed_smem_bytes(int n, bool c_in_smem) { return mix_smem(n, c_in_smem); }
size_t jacobi_mixed_c_bytes(int n) { return (size_t)n * mldc(n) * 4; }

// Rotation slot k of round r (0 <= r < M = npad - 1) of the round-robin
// tournament: the same pairs as jac_pair_of, with the modulo reduced to one
// conditional correction (r + k < 2M, r - k > -M).  The pair comes in
// tournament order (a = r + k + 1, b = r - k + 1, both mod M), not sorted: over
// consecutive slots a counts up and b down, which the layout of A turns into
// distinct banks.
__device__ __forceinline__ void mix_pair(int r, int k, int M, int &a, int &b)
{
    a = 0;
    b = 1 + r;
    if (k != 0) {
        a = r + k;
        if (a >= M) a -= M;
        ++a;
        b = r - k;
        if (b < 0) b += M;
        ++b;
    }
}

// Launch bound 1024 threads, one CTA per SM (the shared memory holds one
// matrix per SM at the sizes that need many threads): the rounds are bound by
// latency, and more warps keep more block updates and eigenvector rotations in
// flight.  The autotuner picks the CTA size per matrix size.
template <bool C_SMEM>
__global__ void __launch_bounds__(2 * kMixMaxThreads, 1) k_jacobi_mixed(const ChanDev *chans, const int *work_ch, int n_work_ch,
                                                               int sample0, int n_terms, const double *coeffs,
                                                               double *lam_s, double *X_s, float *Cf_s,
                                                               double *H_s, int *status_all, int n_ch_total, int *err)
{
    const int wc = blockIdx.x % n_work_ch;
    const int smp = sample0 + blockIdx.x / n_work_ch;
    const int cidx = work_ch[wc];
    const ChanDev ch = chans[cidx];
    const int n = ch.n, N = ch.N, npad = mpad(n), h = npad / 2, M = npad - 1, ldc = mldc(n);
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    if ((size_t)dyn_smem_bytes() < mix_smem(n, C_SMEM)) {
        if (tid == 0) {
            status_all[(size_t)smp * n_ch_total + cidx] = -1;
            record_error(err, kDevBadSize);
        }
        return;
    }
    extern __shared__ float4 smem_f4[];
    unsigned char *sb = reinterpret_cast<unsigned char *>(smem_f4);
    float *A = reinterpret_cast<float *>(sb);
    // one 16-byte record a slot (one shared-memory load): the rotation of the pair (a, b) in
    // tournament order, J = [[c, s'], [-s', c]] on (a, b), s' = s when a < b and -s otherwise
    // (the rotation of the sorted pair (p, q) seen with its indices swapped), then a | b << 16
    // and the column starts mcol(a) | mcol(b) << 16 (A has fewer than 2^16 floats)
    uint4 *rec = reinterpret_cast<uint4 *>(A + mix_a_floats(n));
    float *daa = reinterpret_cast<float *>(rec + h), *dbb = daa + h;
    // flags: [0] rotation in this sweep; [1..3] rotation in this round and [4..6] the
    // round's count of rotating slots, both cycled over three rounds
    int *flags = reinterpret_cast<int *>(dbb + h);
    int *rank = flags + 8;                                            // [h]: index in act, or -1
    unsigned short *act = reinterpret_cast<unsigned short *>(rank + h);  // [h]: the rotating slots
    unsigned short *quad = act + ((h + 1) & ~1);
    const int nq = mquads(n);
    const size_t c_off = ((size_t)(reinterpret_cast<unsigned char *>(quad + ((nq + 1) & ~1)) - sb) + 15) & ~(size_t)15;
    float *C = C_SMEM ? reinterpret_cast<float *>(sb + c_off) : Cf_s + (size_t)blockIdx.x * n * ldc;
    const double *cf = coeffs ? coeffs + (size_t)smp * (n_terms - 1) : nullptr;

    // ---- H in FP64, rounded to FP32; the FP64 H also goes to H_s for the refinement
    double *Hg = H_s ? H_s + (size_t)blockIdx.x * n * n : nullptr;
    for (int e = tid; e < n * n; e += nt) {
        int i = e / n, j = e - i * n;
        if (i > j) continue;
        double v = ch.V[e];
        for (int a = 1; a < n_terms; ++a) v = fma(cf[a - 1], ch.V[(size_t)a * n * n + e], v);
        if (i == j) v += ch.d0 ? ch.d0[i] : ch.h0[i % N];  // d0: the diagonal of a rotated basis
        A[mcol(j) + i] = (float)v;
        if (Hg) {
            Hg[e] = v;
            Hg[(size_t)j * n + i] = v;
        }
    }
    if (npad > n)  // odd n: the phantom index n pairs with a zero row and column, so its rotation is the identity
        for (int i = tid; i <= n; i += nt) A[mcol(n) + i] = 0.0f;
    for (int e = tid; e < n * ldc; e += nt) {
        const int col = e / ldc, row = e - col * ldc;
        C[e] = (row == col) ? 1.0f : 0.0f;  // rows n .. ldc-1 stay zero
    }
    for (int e = tid; e < h * h; e += nt) {  // slot pairs in row order of P
        const int P = e / h, P2 = e - P * h;
        if (P < P2) quad[P * h - P * (P + 1) / 2 + (P2 - P - 1)] = (unsigned short)((P << 8) | P2);
    }
    if (tid < 8) flags[tid] = 0;
    __syncthreads();
    const int nwarps = nt >> 5, warp = tid >> 5;

    // 2 x 2 block B of A in rows (a, b) of the slot of record r1 and columns (a, b) of the slot
    // of record r2: J_1^T B J_2
    auto quad_update = [&](const uint4 r1, const uint4 r2) {
        const int ua = (int)(r1.z & 0xFFFFu), ub = (int)(r1.z >> 16), va = (int)(r2.z & 0xFFFFu), vb = (int)(r2.z >> 16);
        const int sua = (int)(r1.w & 0xFFFFu), sub = (int)(r1.w >> 16), sva = (int)(r2.w & 0xFFFFu), svb = (int)(r2.w >> 16);
        // element (x, y) at mcol(max) + min
        const int i00 = ua <= va ? sva + ua : sua + va;
        const int i01 = ua <= vb ? svb + ua : sua + vb;
        const int i10 = ub <= va ? sva + ub : sub + va;
        const int i11 = ub <= vb ? svb + ub : sub + vb;
        const float b00 = A[i00], b01 = A[i01], b10 = A[i10], b11 = A[i11];
        const float c = __uint_as_float(r1.x), s = __uint_as_float(r1.y);
        const float c2 = __uint_as_float(r2.x), s2 = __uint_as_float(r2.y);
        const float x00 = c2 * b00 - s2 * b01, x01 = s2 * b00 + c2 * b01;
        const float x10 = c2 * b10 - s2 * b11, x11 = s2 * b10 + c2 * b11;
        A[i00] = c * x00 - s * x10;
        A[i01] = c * x01 - s * x11;
        A[i10] = s * x00 + c * x10;
        A[i11] = s * x01 + c * x11;
    };

    int sweeps = 0, g3 = 0;  // g3: the round's flag, cycling over three so a reset never races a read
    bool converged = false;
    while (sweeps < kMixMaxSweeps) {
        if (tid == 0) flags[0] = 0;
        __syncthreads();
        float thr = 0.0f;
        if (n >= kMixThreshN && sweeps < kMixThreshSweeps) {
            float o2 = 0.0f;  // columns j and n - 1 - j per thread: balanced lengths
            for (int j = tid; j < (n + 1) / 2; j += nt) {
                const int jb = mcol(j), j2 = n - 1 - j, j2b = mcol(j2);
                for (int i = 0; i < j; ++i) o2 = fmaf(A[jb + i], A[jb + i], o2);
                if (j2 != j)
                    for (int i = 0; i < j2; ++i) o2 = fmaf(A[j2b + i], A[j2b + i], o2);
            }
            for (int o = 16; o > 0; o >>= 1) o2 += __shfl_xor_sync(0xffffffffu, o2, o);
            if (lane == 0) daa[tid >> 5] = o2;  // daa is free until this sweep's first round
            __syncthreads();
            float tot = 0.0f;
            for (int w = 0; w < (nt >> 5); ++w) tot += daa[w];
            thr = kMixThreshFrac * sqrtf(tot) / (float)n;
            __syncthreads();
        }
        ++sweeps;
        for (int r = 0; r < M; ++r) {
            const int nx3 = g3 == 2 ? 0 : g3 + 1;
            if (tid == 0) {  // last read two rounds ago, before this round's barrier
                flags[1 + nx3] = 0;
                flags[4 + nx3] = 0;
            }
            for (int k = tid; k < h; k += nt) {
                int a, b;
                mix_pair(r, k, M, a, b);
                const bool ab = a < b;
                const int p = ab ? a : b, q = ab ? b : a;
                const int ca = mcol(a), cb = mcol(b), pb = ab ? ca : cb, qb = ab ? cb : ca;
                float c = 1.0f, s = 0.0f, app = A[pb + p], aqq = A[qb + q];
                const float apq = A[qb + p];
                if (fabsf(apq) > kRelTol * sqrtf(fabsf(app) * fabsf(aqq)) && fabsf(apq) > thr) {
                    const float tau = (aqq - app) / (2.0f * apq);
                    float t;
                    if (fabsf(tau) > 1e18f) t = 0.5f / tau;
                    else t = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
                    c = 1.0f / sqrtf(1.0f + t * t);
                    s = t * c;
                    app -= t * apq;
                    aqq += t * apq;
                    flags[0] = 1;
                    flags[1 + g3] = 1;
                    const int idx = atomicAdd(&flags[4 + g3], 1);
                    act[idx] = (unsigned short)k;
                    rank[k] = idx;
                } else {
                    rank[k] = -1;
                }
                rec[k] = make_uint4(__float_as_uint(c), __float_as_uint(ab ? s : -s), (unsigned)a | ((unsigned)b << 16),
                                    (unsigned)ca | ((unsigned)cb << 16));
                daa[k] = ab ? app : aqq;
                dbb[k] = ab ? aqq : app;
            }
            __syncthreads();
            const int na = flags[4 + g3];  // rotating slots this round (the same value for every thread)
            if (na > 0) {
                if (2 * na >= h) {
                    // most slots rotate: every slot pair from the table
                    for (int e = tid; e < nq; e += nt) {
                        const unsigned pr = quad[e];
                        const uint4 r1 = rec[pr >> 8], r2 = rec[pr & 0xFF];
                        // both rotations the identity (s' = +-0)
                        if (__uint_as_float(r1.y) == 0.0f && __uint_as_float(r2.y) == 0.0f) continue;
                        quad_update(r1, r2);
                    }
                } else {
                    // few slots rotate (late sweeps, threshold sweeps): only the pairs that
                    // hold a rotating slot, one warp per rotating slot P, lanes over the
                    // others, rows from P's pair; a pair of two rotating slots is done
                    // once, by the lower one's warp.  A pair with a non-rotating slot
                    // gives the same bits in either orientation (the identity's c = 1,
                    // s' = +-0 leave its side exact), so the result does not depend on
                    // the order of the rotating list.
                    for (int i = warp; i < na; i += nwarps) {
                        const int P = act[i];
                        const uint4 r1 = rec[P];
                        for (int P2 = lane; P2 < h; P2 += 32) {
                            if (P2 == P || (P2 < P && rank[P2] >= 0)) continue;
                            quad_update(r1, rec[P2]);
                        }
                    }
                }
                for (int i = tid; i < na; i += nt) {
                    const int k = act[i];
                    const uint4 rk = rec[k];
                    const int a = (int)(rk.z & 0xFFFFu), b = (int)(rk.z >> 16);
                    const int ca = (int)(rk.w & 0xFFFFu), cb = (int)(rk.w >> 16);
                    A[ca + a] = daa[k];
                    A[cb + b] = dbb[k];
                    A[a < b ? cb + a : ca + b] = 0.0f;
                }
                // C is column-major (column s contiguous, stride ldc): one warp per
                // rotation, each lane four consecutive rows of the two columns
                const int nv = ldc >> 2;
                for (int i = warp; i < na; i += nwarps) {
                    // columns a and b of C: C_a <- c C_a - s' C_b, C_b <- s' C_a + c C_b
                    const uint4 rk = rec[act[i]];
                    float4 *Cp = reinterpret_cast<float4 *>(C + (size_t)(rk.z & 0xFFFFu) * ldc);
                    float4 *Cq = reinterpret_cast<float4 *>(C + (size_t)(rk.z >> 16) * ldc);
                    const float c = __uint_as_float(rk.x), s = __uint_as_float(rk.y);
                    if (!C_SMEM && nv <= 96) {
                        // columns in global memory (L2): every load of the two columns is
                        // issued before the first store, one L2 round trip per rotation
                        float4 a[3], b[3];
#pragma unroll
                        for (int t = 0; t < 3; ++t) {
                            const int v = lane + 32 * t;
                            if (v < nv) {
                                a[t] = Cp[v];
                                b[t] = Cq[v];
                            }
                        }
#pragma unroll
                        for (int t = 0; t < 3; ++t) {
                            const int v = lane + 32 * t;
                            if (v < nv) {
                                Cp[v] = make_float4(c * a[t].x - s * b[t].x, c * a[t].y - s * b[t].y,
                                                    c * a[t].z - s * b[t].z, c * a[t].w - s * b[t].w);
                                Cq[v] = make_float4(s * a[t].x + c * b[t].x, s * a[t].y + c * b[t].y,
                                                    s * a[t].z + c * b[t].z, s * a[t].w + c * b[t].w);
                            }
                        }
                        continue;
                    }
                    for (int v = lane; v < nv; v += 32) {
                        const float4 a = Cp[v], b = Cq[v];
                        Cp[v] = make_float4(c * a.x - s * b.x, c * a.y - s * b.y, c * a.z - s * b.z, c * a.w - s * b.w);
                        Cq[v] = make_float4(s * a.x + c * b.x, s * a.y + c * b.y, s * a.z + c * b.z, s * a.w + c * b.w);
                    }
                }
                __syncthreads();
            }
            g3 = nx3;
        }
        if (flags[0] == 0 && thr == 0.0f) {  // a thresholded sweep proves nothing
            converged = true;
            break;
        }
        __syncthreads();
    }

    // ---- FP32 eigenpairs out, as FP64, unsorted
    double *X = X_s + (size_t)blockIdx.x * n * n;  // row-major out of the column-major C
    for (int e = tid; e < n * n; e += nt) {
        const int col = e / n, row = e - col * n;
        X[(size_t)row * n + col] = (double)C[(size_t)col * ldc + row];
    }
    for (int i = tid; i < n; i += nt) lam_s[(size_t)blockIdx.x * n + i] = (double)A[mcol(i) + i];
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
    const bool cs = mix_smem(n, true) <= kMixSmemCap;
    if (threads < 32 || threads > 2 * kMixMaxThreads || (threads & 31)) return cudaErrorInvalidValue;
    const size_t smem = mix_smem(n, cs);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    dim3 grid((unsigned)(n_samples * n_work_ch));
    if (cs) {
        raise_smem_limit((const void *)k_jacobi_mixed<true>, smem);
        k_jacobi_mixed<true><<<grid, threads, smem, counted(st)>>>(chans_dev, work_ch_dev, n_work_ch, sample0, n_terms,
                                                              coeffs, lam_s, X_s, Cf_s, H_s, status_all, n_ch_total, err);
    } else {
        raise_smem_limit((const void *)k_jacobi_mixed<false>, smem);
        k_jacobi_mixed<false><<<grid, threads, smem, counted(st)>>>(chans_dev, work_ch_dev, n_work_ch, sample0, n_terms,
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
        raise_smem_limit((const void *)k_jacobi_mixed<true>, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_jacobi_mixed<true>, threads, smem);
    } else {
        raise_smem_limit((const void *)k_jacobi_mixed<false>, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_jacobi_mixed<false>, threads, smem);
    }
    return blocks;
}

}  // namespace wpcd
