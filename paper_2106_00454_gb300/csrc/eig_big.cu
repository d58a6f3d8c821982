// eig_big.cu -- (a2, a3) parameter sum + symmetric eigensolve for matrices too
// large for one CTA's shared memory (Sec. 3.2 step 2; the paper's GPU code was
// limited to shared-memory-sized matrices, App. C and Sec. 7).
//
// The same parallel cyclic two-sided Jacobi method as the shared-memory
// kernels (round-robin tournament: each round applies npad/2 disjoint
// rotations, every pair once per sweep), with the matrix and the eigenvectors
// in global memory, where they stay L2-resident while the CTA works on them.
// Jacobi is kept at every size because the spectrum of H = H0 + V is graded
// (eigenvalues from ~1e-10 to ~10 fm^-1) and the resolvent needs the small
// ones to their own relative accuracy; a Householder reduction in FP32 does
// not deliver that.
//
// Storage, per item (one item = one (sample, channel) solve), in a scratch
// slot of the launch (the grid strides over the items):
//   A  [npad][npad] T, the full symmetric matrix, row-major; odd n carries a
//      zero phantom row and column n, whose rotation is always the identity;
//   Cc [npad][npad] T, the eigenvectors column by column (vector s contiguous).
// A round is two phases:
//   1. every slot k computes its rotation (c_k, s_k) from (a_pp, a_qq, a_pq);
//   2. warp w takes the row pairs P = w, w + nwarps, ...: for every column
//      slot P2 its lanes replace the 2 x 2 block A[{p,q}][{p2,q2}] by
//      J_P^T B J_P2 (rows p, q read and written whole, lane-contiguous along
//      the slot order, so the accesses coalesce); the diagonal blocks become
//      (a_pp', 0; 0, a_qq').  The same phase rotates columns p, q of Cc.
// Different row pairs touch disjoint rows, so phase 2 needs no atomics.
//
// FP64 (T = double): a pair rotates whenever a_pq != 0; sweeps stop when
// off(A) <= 1e-15 ||H||_F (as the shared-memory FP64 kernel).  Eigenvalues
// leave sorted ascending, eigenvectors permuted alike, in the eigen-buffer
// layout (row-major C[row][s]).
// FP32 (T = float, mixed precision): H formed in FP64 (also written out for
// the FP64 refinement) and rounded to FP32; the relative rotation test
// |a_pq| > 2^-23 sqrt|a_pp a_qq| (plus a threshold in the first two sweeps);
// sweeps stop after a sweep without rotations.  Eigenpairs leave unsorted as
// FP64 in the refinement's layout.
#include <math.h>

#include "wpcd_internal.cuh"

namespace wpcd {

constexpr int kBigThreads = 512;
constexpr int kBigMaxSweeps = 40;
constexpr int kBigMaxN = 2 * kMaxNwp;
constexpr float kBigRelTol = 1.1920929e-7f;  // 2^-23
constexpr int kBigThreshSweeps = 2;
constexpr float kBigThreshFrac = 0.1f;
// column slots (or eigenvector rows) whose loads a lane batches: 8 in FP32, 4 in FP64 (registers)
template <class T>
struct BigUnroll {
    static constexpr int v = sizeof(T) == 8 ? 4 : 8;
};

__host__ __device__ inline int big_pad(int n) { return (n + 1) & ~1; }

template <class T>
__host__ __device__ inline size_t big_slot_elems(int n)
{
    const size_t np = (size_t)big_pad(n);
    return 2 * np * np;  // A and Cc
}

template <class T>
struct BigRot {
    T c, s, app, aqq;
};

// Rotation slot k of round r: the pair (a, b) in tournament order (a runs up
// with k, b down, so consecutive slots touch consecutive columns), p < q.
__device__ __forceinline__ void big_pair(int r, int k, int M, int &a, int &b)
{
    if (k == 0) {
        a = 0;
        b = 1 + r;
    } else {
        a = r + k;
        if (a >= M) a -= M;
        ++a;
        b = r - k;
        if (b < 0) b += M;
        ++b;
    }
}

template <class T>
__device__ __forceinline__ T big_abs(T x) { return x < T(0) ? -x : x; }

// (o1, o2) = (c u - s v, s u + c v), with the roundings spelled out so that the
// two warps that compute an off-diagonal block and its mirror image (in
// opposite rotation order, below) produce bit-identical results.
__device__ __forceinline__ void big_rot(float c, float s, float u, float v, float &o1, float &o2)
{
    o1 = fmaf(c, u, -__fmul_rn(s, v));
    o2 = fmaf(s, u, __fmul_rn(c, v));
}
__device__ __forceinline__ void big_rot(double c, double s, double u, double v, double &o1, double &o2)
{
    o1 = fma(c, u, -__dmul_rn(s, v));
    o2 = fma(s, u, __dmul_rn(c, v));
}

template <class T>
__global__ void __launch_bounds__(kBigThreads, 1) k_jacobi_big(const ChanDev *chans, const int *work_ch, int n_work_ch,
                                                          int n_items, int sample0, int n_terms, const double *coeffs,
                                                          T *scratch, double *eps_all, double *C_all, double *lam_s,
                                                          double *X_s, double *H_s, int *status_all, int n_ch_total,
                                                          int *err)
{
    constexpr bool F64 = sizeof(T) == 8;
    constexpr int kBigUnroll = BigUnroll<T>::v;
    extern __shared__ double smem_big[];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int wc = item % n_work_ch;
        const int smp = sample0 + item / n_work_ch;
        const int cidx = work_ch[wc];
        const ChanDev ch = chans[cidx];
        const int n = ch.n, N = ch.N, np = big_pad(n), h = np / 2, M = np - 1;
        // per-round tables in shared memory: slots {p, q, a, b} and rotations
        int4 *sl = reinterpret_cast<int4 *>(smem_big);
        BigRot<T> *rot = reinterpret_cast<BigRot<T> *>(sl + h);
        double *red = reinterpret_cast<double *>(rot + h);  // 32 doubles
        // flag: [0] rotation this sweep; [1..3] rotating slots this round, cycled over three rounds
        int *flag = reinterpret_cast<int *>(red + 32);
        int *act = flag + 4;   // [h] the round's rotating slots
        int *rank = act + h;   // [np] eigenvalue ranks for the final sort
        const size_t need = (size_t)h * (sizeof(int4) + sizeof(BigRot<T>)) + 32 * 8 + 4 * 4 + (size_t)h * 4 +
                            (size_t)np * 4;
        if (n > kBigMaxN || (size_t)dyn_smem_bytes() < need) {
            if (tid == 0) {
                status_all[(size_t)smp * n_ch_total + cidx] = -1;
                record_error(err, kDevBadSize);
            }
            continue;
        }
        T *A = scratch + (size_t)blockIdx.x * big_slot_elems<T>(n);
        T *Cc = A + (size_t)np * np;
        const double *cf = coeffs ? coeffs + (size_t)smp * (n_terms - 1) : nullptr;
        double *Hg = (!F64 && H_s) ? H_s + (size_t)item * n * n : nullptr;

        // ---- (a2) H = diag(H0) + V0 + sum_a c_a V_a (full matrix), and Cc = I
        double fro2 = 0.0;
        for (int e = tid; e < np * np; e += nt) {
            const int i = e / np, j = e - i * np;
            double v = 0.0;
            if (i < n && j < n) {
                // the upper triangle's value on both sides: H exactly symmetric
                const size_t ij = i <= j ? (size_t)i * n + j : (size_t)j * n + i;
                v = ch.V[ij];
                for (int a = 1; a < n_terms; ++a) v = fma(cf[a - 1], ch.V[(size_t)a * n * n + ij], v);
                if (i == j) v += ch.d0 ? ch.d0[i] : ch.h0[i % N];  // d0: the diagonal of a rotated basis
                if (Hg) Hg[(size_t)i * n + j] = v;
                fro2 = fma(v, v, fro2);
            }
            A[e] = (T)v;
            Cc[e] = (i == j) ? T(1) : T(0);
        }
        fro2 = cta_sum64(fro2, red);
        if (tid < 4) flag[tid] = 0;
        __syncthreads();
        const double tol2 = 1e-30 * fro2;  // FP64 stop: (1e-15 ||H||_F)^2

        int sweeps = 0, g3 = 0;
        bool converged = false;
        while (sweeps < kBigMaxSweeps) {
            T thr = T(0);
            if (F64 || (sweeps < kBigThreshSweeps)) {
                // off(A)^2 over the strict upper triangle (FP64 stop test; FP32 threshold)
                double o2 = 0.0;
                for (int i = warp; i < n; i += nwarp)
                    for (int j = i + 1 + lane; j < n; j += 32) {
                        const double x = (double)A[(size_t)i * np + j];
                        o2 = fma(x, x, o2);
                    }
                o2 = cta_sum64(o2, red);
                if (F64) {
                    if (2.0 * o2 <= tol2) {
                        converged = true;
                        break;
                    }
                } else {
                    thr = (T)(kBigThreshFrac * sqrt(o2) / n);
                }
            }
            if (tid == 0) flag[0] = 0;
            __syncthreads();
            ++sweeps;
            for (int r = 0; r < M; ++r) {
                const int nx3 = g3 == 2 ? 0 : g3 + 1;
                if (tid == 0) flag[1 + nx3] = 0;  // last read two rounds ago
                // phase 1: the rotations of this round
                for (int k = tid; k < h; k += nt) {
                    int a, b;
                    big_pair(r, k, M, a, b);
                    const int p = a < b ? a : b, q = a < b ? b : a;
                    T c = T(1), s = T(0), app = A[(size_t)p * np + p], aqq = A[(size_t)q * np + q];
                    const T apq = A[(size_t)p * np + q];
                    bool rotate;
                    if (F64) rotate = apq != T(0);
                    else rotate = big_abs(apq) > (T)kBigRelTol * sqrt(big_abs(app) * big_abs(aqq)) && big_abs(apq) > thr;
                    if (rotate) {
                        const T tau = (aqq - app) / (T(2) * apq);
                        T t;
                        if (big_abs(tau) > (F64 ? T(1e150) : T(1e18))) t = T(0.5) / tau;
                        else t = (tau >= T(0) ? T(1) : T(-1)) / (big_abs(tau) + sqrt(T(1) + tau * tau));
                        c = T(1) / sqrt(T(1) + t * t);
                        s = t * c;
                        app -= t * apq;
                        aqq += t * apq;
                        flag[0] = 1;
                        act[atomicAdd(&flag[1 + g3], 1)] = k;
                    }
                    sl[k] = make_int4(p, q, a, b);
                    rot[k] = BigRot<T>{c, s, app, aqq};
                }
                __syncthreads();
                const int na = flag[1 + g3];  // rotating slots this round
                if (na > 0) {
                    // phase 2: rows p, q of every row pair, and columns p, q of Cc.  Each lane
                    // issues the loads of kBigUnroll column slots (or rows of Cc) before any
                    // store: the accesses are L2 round trips, and a store may alias a later
                    // load for all the compiler knows, so batching them is what keeps
                    // enough requests in flight
                    for (int P = warp; P < h; P += nwarp) {
                        const int4 u = sl[P];
                        const BigRot<T> r1 = rot[P];
                        T *Rp = A + (size_t)u.x * np, *Rq = A + (size_t)u.y * np;
                        // a rotating row pair meets every column slot; a fixed one only the
                        // rotating slots (the other blocks stay as they are)
                        const bool pa_rot = r1.s != T(0);
                        const int kend = pa_rot ? h : na;
                        for (int k0 = lane; k0 < kend; k0 += 32 * kBigUnroll) {
                            T pa[kBigUnroll], pb[kBigUnroll], qa[kBigUnroll], qb[kBigUnroll];
                            int ca[kBigUnroll], cb[kBigUnroll], kk[kBigUnroll];
                            bool on[kBigUnroll];
#pragma unroll
                            for (int t = 0; t < kBigUnroll; ++t) {
                                const int j = k0 + 32 * t;
                                const int k = j < kend ? (pa_rot ? j : act[j]) : 0;
                                kk[t] = k;
                                on[t] = j < kend && k != P && !(r1.s == T(0) && rot[k].s == T(0));
                                if (on[t]) {
                                    const int4 v = sl[k];
                                    ca[t] = v.z;
                                    cb[t] = v.w;
                                    pa[t] = Rp[v.z];
                                    pb[t] = Rp[v.w];
                                    qa[t] = Rq[v.z];
                                    qb[t] = Rq[v.w];
                                }
                            }
#pragma unroll
                            for (int t = 0; t < kBigUnroll; ++t) {
                                if (!on[t]) continue;
                                const int k = kk[t];
                                const BigRot<T> r2 = rot[k];
                                // columns in slot order (a, b); the rotation acts on (p2, q2) = (min, max)
                                const bool ab = ca[t] < cb[t];
                                const T b00 = ab ? pa[t] : pb[t], b01 = ab ? pb[t] : pa[t];
                                const T b10 = ab ? qa[t] : qb[t], b11 = ab ? qb[t] : qa[t];
                                // J_P^T B J_k, the rotation of the lower slot index applied first:
                                // the mirror block (rows of slot k, columns of slot P) is then the
                                // exact transpose, and A stays exactly symmetric
                                T y00, y01, y10, y11;
                                if (k > P) {
                                    T x00, x01, x10, x11;
                                    big_rot(r2.c, r2.s, b00, b01, x00, x01);  // columns (J_k)
                                    big_rot(r2.c, r2.s, b10, b11, x10, x11);
                                    big_rot(r1.c, r1.s, x00, x10, y00, y10);  // rows (J_P)
                                    big_rot(r1.c, r1.s, x01, x11, y01, y11);
                                } else {
                                    T z00, z01, z10, z11;
                                    big_rot(r1.c, r1.s, b00, b10, z00, z10);  // rows (J_P)
                                    big_rot(r1.c, r1.s, b01, b11, z01, z11);
                                    big_rot(r2.c, r2.s, z00, z01, y00, y01);  // columns (J_k)
                                    big_rot(r2.c, r2.s, z10, z11, y10, y11);
                                }
                                Rp[ca[t]] = ab ? y00 : y01;
                                Rp[cb[t]] = ab ? y01 : y00;
                                Rq[ca[t]] = ab ? y10 : y11;
                                Rq[cb[t]] = ab ? y11 : y10;
                            }
                        }
                        if (r1.s != T(0)) {
                            if (lane == 0) {  // the diagonal block of the pair
                                Rp[u.x] = r1.app;
                                Rq[u.y] = r1.aqq;
                                Rp[u.y] = T(0);
                                Rq[u.x] = T(0);
                            }
                            T *Cp = Cc + (size_t)u.x * np, *Cq = Cc + (size_t)u.y * np;
                            for (int r0 = lane; r0 < np; r0 += 32 * kBigUnroll) {
                                T a[kBigUnroll], b[kBigUnroll];
#pragma unroll
                                for (int t = 0; t < kBigUnroll; ++t) {
                                    const int row = r0 + 32 * t;
                                    if (row < np) {
                                        a[t] = Cp[row];
                                        b[t] = Cq[row];
                                    }
                                }
#pragma unroll
                                for (int t = 0; t < kBigUnroll; ++t) {
                                    const int row = r0 + 32 * t;
                                    if (row < np) {
                                        T x, y;
                                        big_rot(r1.c, r1.s, a[t], b[t], x, y);
                                        Cp[row] = x;
                                        Cq[row] = y;
                                    }
                                }
                            }
                        }
                    }
                    __syncthreads();
                }
                g3 = nx3;
            }
            if (!F64) {
                if (flag[0] == 0 && thr == T(0)) {  // a thresholded sweep proves nothing
                    converged = true;
                    break;
                }
                __syncthreads();
            }
        }

        if (F64) {
            // eigenvalues ascending (rank sort, ties by index), eigenvectors permuted alike
            double *eps = eps_all + ch.eps_off + (size_t)smp * n;
            double *Cg = C_all + ch.c_off + (size_t)smp * n * n;
            for (int i = tid; i < n; i += nt) {
                const double ei = (double)A[(size_t)i * np + i];
                int rk = 0;
                for (int j = 0; j < n; ++j) {
                    const double ej = (double)A[(size_t)j * np + j];
                    rk += (ej < ei) || (ej == ei && j < i);
                }
                rank[i] = rk;
                eps[rk] = ei;
            }
            __syncthreads();
            for (int s = warp; s < n; s += nwarp) {
                const int cs = rank[s];
                for (int row = lane; row < n; row += 32) Cg[(size_t)row * n + cs] = (double)Cc[(size_t)s * np + row];
            }
        } else {
            double *X = X_s + (size_t)item * n * n;  // row-major, unsorted
            for (int s = warp; s < n; s += nwarp)
                for (int row = lane; row < n; row += 32) X[(size_t)row * n + s] = (double)Cc[(size_t)s * np + row];
            for (int i = tid; i < n; i += nt) lam_s[(size_t)item * n + i] = (double)A[(size_t)i * np + i];
        }
        if (tid == 0) {
            status_all[(size_t)smp * n_ch_total + cidx] = converged ? sweeps : -1;
            if (!converged) record_error(err, kDevNoConverge);
        }
        __syncthreads();  // the slot's scratch and tables are reused by the next item
    }
}

template <class T>
static size_t big_smem(int n)
{
    const int np = big_pad(n), h = np / 2;
    return (size_t)h * (sizeof(int4) + sizeof(BigRot<T>)) + 32 * 8 + 4 * 4 + (size_t)h * 4 + (size_t)np * 4;
}

// Whether the shared-memory kernel of that precision holds an n x n matrix
// (its packed matrix and round tables in one CTA's 227 KB, eigenvectors in
// global memory if need be); above that the global-memory kernel runs.
bool jacobi_fits_smem(int n, bool f64)
{
    const size_t cap = 227 * 1024;
    return f64 ? jacobi_smem_bytes(n, false) <= cap : jacobi_mixed_smem_bytes(n, false) <= cap;
}

size_t jacobi_big_scratch_bytes(int n, bool f64) { return big_slot_elems<double>(n) * (f64 ? 8 : 4); }

int jacobi_big_max_n() { return kBigMaxN; }

// Resident CTAs per SM of the large-matrix kernel (the grid strides over items).
int jacobi_big_occupancy(int n, bool f64)
{
    int blocks = 0;
    if (f64) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_jacobi_big<double>, kBigThreads, big_smem<double>(n));
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_jacobi_big<float>, kBigThreads, big_smem<float>(n));
    return blocks;
}

// FP64: eigenpairs into the eigen buffer (eps_all / C_all at the channel offsets).
// FP32: lam_s [item][n], X_s [item][n][n] and H_s [item][n][n] in the refinement layout.
// scratch: `slots` slots of jacobi_big_scratch_bytes(n, f64) bytes; the grid has
// min(items, slots) CTAs, each working through items with the grid's stride.
cudaError_t launch_jacobi_big(bool f64, const ChanDev *chans_dev, const int *work_ch_dev, int n_work_ch,
                              int n_samples, int sample0, int n_terms, const double *coeffs, int n, void *scratch,
                              int slots, double *eps_all, double *C_all, double *lam_s, double *X_s, double *H_s,
                              int *status_all, int n_ch_total, int *err, cudaStream_t st)
{
    if (n < 2 || n > kBigMaxN || slots < 1) return cudaErrorInvalidValue;
    const int items = n_samples * n_work_ch;
    const int grid = items < slots ? items : slots;
    if (f64) {
        const size_t sm = big_smem<double>(n);
        raise_smem_limit((const void *)k_jacobi_big<double>, sm);
        k_jacobi_big<double><<<grid, kBigThreads, sm, counted(st)>>>(
            chans_dev, work_ch_dev, n_work_ch, items, sample0, n_terms, coeffs, static_cast<double *>(scratch), eps_all,
            C_all, nullptr, nullptr, nullptr, status_all, n_ch_total, err);
    } else {
        const size_t sm = big_smem<float>(n);
        raise_smem_limit((const void *)k_jacobi_big<float>, sm);
        k_jacobi_big<float><<<grid, kBigThreads, sm, counted(st)>>>(
            chans_dev, work_ch_dev, n_work_ch, items, sample0, n_terms, coeffs, static_cast<float *>(scratch), nullptr,
            nullptr, lam_s, X_s, H_s, status_all, n_ch_total, err);
    }
    return cudaGetLastError();
}

}  // namespace wpcd
