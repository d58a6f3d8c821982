// mi.cu -- matrix-inversion (MI) solution of the LS equation (Sec. 2.1), the
// paper's comparison method, batched over (sample, channel, energy).
//
// The real K-matrix with the Haftel-Tabakin pole subtraction on the grid
// {k_j} (N_Q Gauss-Legendre points mapped by k = c tan(pi (1 + x) / 4)) plus
// the on-shell point p:
//   D_j = w_j k_j^2 2 mu / (p^2 - k_j^2)  (j < N_Q),
//   D_N = -2 mu p^2 sum_j w_j / (p^2 - k_j^2),
//   (1 - V D) K = V,
// with the on-shell K, T = (1 + i pi mu p K)^-1 K, S = 1 - 2 pi i mu p T and
// the phases.  As in the paper's timing study (Sec. 6) the equation is solved
// at n_I interpolation energies and the phase shifts are interpolated linearly
// in T_lab to the requested energies, from which the np total cross section
// follows.
//
// GB300 layout: the potential terms on the grid are computed once per channel
// set (k_mi_pot_grid) and the on-shell rows once per energy list
// (k_mi_pot_onshell); k_mi_solve runs persistent CTAs, each owning a slot of
// FP64 scratch for one (sample, channel) matrix V = V0 + sum_a c_a V_a, and for
// every energy inverts 1 - V D in FP32 in shared memory (Gauss-Jordan, partial
// pivoting; FP32 issues at 58x the FP64 rate) and refines the solution to FP64
// accuracy with FP64 residuals r = b - (x - V (D x)) (classical iterative
// refinement: every step is two matrix-vector products).
#include <math.h>

#include "potential.cuh"
#include "wpcd_internal.cuh"

namespace wpcd {

constexpr int kMiThreads = 512;  // one CTA per SM for coupled systems: 16 warps to hide latency
constexpr int kMiMaxRefine = 30;

// ------------------------------------------------------------------------------------- grid
__global__ void k_mi_grid(int NQ, double cmap, const double *glx, const double *glw, double *k, double *w)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= NQ) return;
    const double th = kPi * (1.0 + glx[j]) / 4.0, cth = cos(th);
    k[j] = cmap * tan(th);
    w[j] = cmap * (kPi / 4.0) * glw[j] / (cth * cth);
}

cudaError_t launch_mi_grid(int NQ, double cmap, const double *glx, const double *glw, double *k, double *w,
                           cudaStream_t st)
{
    k_mi_grid<<<(NQ + 127) / 128, 128, 0, counted(st)>>>(NQ, cmap, glx, glw, k, w);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------- potential
__device__ __forceinline__ int mi_lblock(const MiChanDev &c, int a)
{
    return c.coupled ? (a == 0 ? c.J - 1 : c.J + 1) : c.l;
}

// Grid part of V_t for every channel: entries (a, i), (b, j) with i, j < N_Q;
// one thread per grid pair i <= j (the mirror follows from V^{l'l}(p', p) =
// V^{ll'}(p, p')).  Vg of channel c: [n_terms][n][n] at c.vg_off, n = K (N_Q+1).
template <int GEN>
__global__ void __launch_bounds__(128) k_mi_pot_grid(const MiChanDev *chans, int n_ch, int NQ, const double *kg,
                                                     int Lmax, const double *gp, const double *angx,
                                                     const double *angw, int n_terms, double *Vg)
{
    __shared__ double wpl[kAngleQ][kLmaxReg + 1];
    __shared__ double ax[kAngleQ];
    const int Lm = (Lmax < kLmaxReg) ? Lmax : kLmaxReg;
    if (GEN == WPCD_GEN_YUKAWA) {
        angle_tables(angx, angw, Lm, wpl, ax);
        __syncthreads();
    }
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (long long)NQ * (NQ + 1) / 2) return;
    int j = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while ((long long)(j + 1) * (j + 2) / 2 <= b) ++j;
    while ((long long)j * (j + 1) / 2 > b) --j;
    const int i = (int)(b - (long long)j * (j + 1) / 2);
    const double pp = kg[i], p = kg[j];
    double I1[kLmaxReg + 1], I2[kLmaxReg + 1], I3[kLmaxReg + 1], R = 0.0;
    if (GEN == WPCD_GEN_YUKAWA) yukawa_angle_integrals(gp, wpl, ax, Lm, pp, p, I1, I2, I3, R);
    const int M = NQ + 1;
    for (int c = 0; c < n_ch; ++c) {
        const MiChanDev ch = chans[c];
        const int n = ch.n;
        for (int al = 0; al < ch.K; ++al)
            for (int be = 0; be < ch.K; ++be) {
                double tv[kMaxTerms];
                potential_terms<GEN>(gp, ch.s, ch.J, ch.tz, mi_lblock(ch, al), mi_lblock(ch, be), pp, p, I1, I2, I3,
                                     R, tv);
                for (int t = 0; t < n_terms; ++t) {
                    double *V = Vg + ch.vg_off + (size_t)t * n * n;
                    V[(size_t)(al * M + i) * n + (be * M + j)] = tv[t];
                    V[(size_t)(be * M + j) * n + (al * M + i)] = tv[t];
                }
            }
    }
}

// On-shell column of V_t at each energy: V_t^{l_a l_b}(q_i, p_e) for q_i = k_i
// (i < N_Q) and q_N = p_e.  Von of channel c: [n_I][n_terms][K][K][N_Q+1] at
// c.von_off.  One thread per (energy, i).
template <int GEN>
__global__ void __launch_bounds__(128) k_mi_pot_onshell(const MiChanDev *chans, int n_ch, int NQ, const double *kg,
                                                        int n_I, const double *e_int, int Lmax, const double *gp,
                                                        const double *angx, const double *angw, int n_terms,
                                                        double *Von)
{
    __shared__ double wpl[kAngleQ][kLmaxReg + 1];
    __shared__ double ax[kAngleQ];
    const int Lm = (Lmax < kLmaxReg) ? Lmax : kLmaxReg;
    if (GEN == WPCD_GEN_YUKAWA) {
        angle_tables(angx, angw, Lm, wpl, ax);
        __syncthreads();
    }
    const int M = NQ + 1;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_I * M) return;
    const int e = b / M, i = b - e * M;
    const double p = sqrt(kMn * e_int[e] / 2.0) / kHbarc;
    const double pp = i < NQ ? kg[i] : p;
    double I1[kLmaxReg + 1], I2[kLmaxReg + 1], I3[kLmaxReg + 1], R = 0.0;
    if (GEN == WPCD_GEN_YUKAWA) yukawa_angle_integrals(gp, wpl, ax, Lm, pp, p, I1, I2, I3, R);
    for (int c = 0; c < n_ch; ++c) {
        const MiChanDev ch = chans[c];
        for (int al = 0; al < ch.K; ++al)
            for (int be = 0; be < ch.K; ++be) {
                double tv[kMaxTerms];
                potential_terms<GEN>(gp, ch.s, ch.J, ch.tz, mi_lblock(ch, al), mi_lblock(ch, be), pp, p, I1, I2, I3,
                                     R, tv);
                for (int t = 0; t < n_terms; ++t)
                    Von[ch.von_off + ((((size_t)e * n_terms + t) * ch.K + al) * ch.K + be) * M + i] = tv[t];
            }
    }
}

cudaError_t launch_mi_pot(int gen, const MiChanDev *chans_dev, int n_ch, int NQ, const double *kg, int Lmax,
                          const double *gp_dev, const double *angx, const double *angw, int n_terms, double *Vg,
                          cudaStream_t st)
{
    const long long pairs = (long long)NQ * (NQ + 1) / 2;
    const unsigned grid = (unsigned)((pairs + 127) / 128);
    if (gen == WPCD_GEN_YUKAWA)
        k_mi_pot_grid<WPCD_GEN_YUKAWA><<<grid, 128, 0, counted(st)>>>(chans_dev, n_ch, NQ, kg, Lmax, gp_dev, angx, angw,
                                                             n_terms, Vg);
    else
        k_mi_pot_grid<WPCD_GEN_YAMAGUCHI><<<grid, 128, 0, counted(st)>>>(chans_dev, n_ch, NQ, kg, 0, gp_dev, nullptr, nullptr,
                                                                n_terms, Vg);
    return cudaGetLastError();
}

cudaError_t launch_mi_onshell(int gen, const MiChanDev *chans_dev, int n_ch, int NQ, const double *kg, int n_I,
                              const double *e_int, int Lmax, const double *gp_dev, const double *angx,
                              const double *angw, int n_terms, double *Von, cudaStream_t st)
{
    const unsigned grid = (unsigned)((n_I * (NQ + 1) + 127) / 128);
    if (gen == WPCD_GEN_YUKAWA)
        k_mi_pot_onshell<WPCD_GEN_YUKAWA><<<grid, 128, 0, counted(st)>>>(chans_dev, n_ch, NQ, kg, n_I, e_int, Lmax, gp_dev, angx,
                                                                angw, n_terms, Von);
    else
        k_mi_pot_onshell<WPCD_GEN_YAMAGUCHI><<<grid, 128, 0, counted(st)>>>(chans_dev, n_ch, NQ, kg, n_I, e_int, 0, gp_dev,
                                                                   nullptr, nullptr, n_terms, Von);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------- solve
// Shared memory of one CTA for matrices up to n: A float [n][ld] | D double [M] |
// b, x, r double [2][n] | y float [2][n] | perm int [n, even] | reduction double [64].
__host__ __device__ inline int mi_ld(int n) { return (n + 3) & ~3; }  // rows padded to 16 bytes (float4 access)

__host__ __device__ inline size_t mi_smem(int n, int M)
{
    size_t a = (size_t)n * mi_ld(n) * 4;
    a = (a + 15) & ~(size_t)15;
    return a + (size_t)M * 8 + 3 * (size_t)2 * n * 8 + (size_t)2 * n * 4 + (size_t)(n + (n & 1)) * 4 + 64 * 8;
}

size_t mi_smem_bytes(int n, int M) { return mi_smem(n, M); }

// Maximum over the CTA that propagates NaN (fmax would drop it).
__device__ __forceinline__ double nan_max(double a, double b) { return (b > a || b != b) ? b : a; }

__device__ __forceinline__ double mi_block_max(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v = nan_max(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = nan_max(t, red[w]);
    return t;
}

__device__ __forceinline__ double mi_block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

// Items (sample, work channel) of one block size; CTA blockIdx.x owns scratch
// slot Vs + blockIdx.x n^2 and walks the items item = blockIdx.x, + gridDim.x, ...
// Outputs per (sample, channel, energy): phases ph [S][n_ch][n_I][3] (degrees)
// and, if k_out, the on-shell K [S][n_ch][n_I][2][2].
__global__ void __launch_bounds__(kMiThreads) k_mi_solve(const MiChanDev *chans, const int *work_ch, int n_work,
                                                         int n_ch_total, int n_samples, int NQ, const double *kg,
                                                         const double *wg, int n_terms, const double *coeffs,
                                                         const double *Vg, const double *Von, int n_I,
                                                         const double *e_int, double *Vs_all, double *ph,
                                                         double *k_out, int *status, int *err)
{
    const int M = NQ + 1;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    if ((size_t)dyn_smem_bytes() < mi_smem(chans[work_ch[0]].n, M)) {  // launch/layout mismatch
        if (tid == 0) record_error(err, kDevBadSize);
        return;
    }
    extern __shared__ __align__(16) double mi_sm[];
    unsigned char *sb = reinterpret_cast<unsigned char *>(mi_sm);
    const int n0 = chans[work_ch[0]].n;  // every work channel of a launch has the same n
    const int ld = mi_ld(n0);
    size_t off = ((size_t)n0 * ld * 4 + 15) & ~(size_t)15;
    float *A = reinterpret_cast<float *>(sb);
    double *D = reinterpret_cast<double *>(sb + off);
    double *bv = D + M, *xv = bv + 2 * n0, *rv = xv + 2 * n0;
    float *yv = reinterpret_cast<float *>(rv + 2 * n0);
    int *perm = reinterpret_cast<int *>(yv + 2 * n0);
    double *red = reinterpret_cast<double *>(perm + n0 + (n0 & 1));
    double *Vs = Vs_all + (size_t)blockIdx.x * 2 * n0 * n0;  // V, then the FP64 fallback matrix

    for (int item = blockIdx.x; item < n_samples * n_work; item += gridDim.x) {
        const int smp = item / n_work, cidx = work_ch[item - smp * n_work];
        const MiChanDev ch = chans[cidx];
        const int n = ch.n, K = ch.K;
        const double *cf = coeffs ? coeffs + (size_t)smp * (n_terms - 1) : nullptr;
        const double *Vgc = Vg + ch.vg_off;
        // V = V0 + sum_a c_a V_a on the grid part (the on-shell rows follow per energy)
        for (int e = tid; e < n * n; e += nt) {
            const int r = e / n, c = e - r * n;
            if (r % M == NQ || c % M == NQ) continue;
            double v = Vgc[e];
            for (int t = 1; t < n_terms; ++t) v = fma(cf[t - 1], Vgc[(size_t)t * n * n + e], v);
            Vs[e] = v;
        }
        int worst = 0;
        for (int ie = 0; ie < n_I; ++ie) {
            const double p = sqrt(kMn * e_int[ie] / 2.0) / kHbarc, p2 = p * p;
            // D and the on-shell rows and columns of V at this energy
            double part = 0.0;
            for (int j = tid; j < NQ; j += nt) {
                const double den = p2 - kg[j] * kg[j];
                D[j] = wg[j] * kg[j] * kg[j] * 2.0 * kMu / den;
                part += wg[j] / den;
            }
            const double sum = mi_block_sum(part, red);
            if (tid == 0) D[NQ] = -2.0 * kMu * p2 * sum;
            const double *Vo = Von + ch.von_off + (size_t)ie * n_terms * K * K * M;
            for (int e = tid; e < K * K * M; e += nt) {
                const int al = e / (K * M), be = (e / M) % K, i = e % M;
                double v = Vo[e];
                for (int t = 1; t < n_terms; ++t) v = fma(cf[t - 1], Vo[(size_t)t * K * K * M + e], v);
                Vs[(size_t)(al * M + i) * n + (be * M + NQ)] = v;  // V^{l_a l_b}(q_i, p)
                Vs[(size_t)(be * M + NQ) * n + (al * M + i)] = v;  // V^{l_b l_a}(p, q_i), the same value
            }
            __syncthreads();
            // A = 1 - V D (FP32), right-hand sides b_bb = V[:, (bb, N)] (FP64)
            for (int e = tid; e < n * n; e += nt) {
                const int r = e / n, c = e - r * n;
                A[(size_t)r * ld + c] = (float)((r == c ? 1.0 : 0.0) - Vs[e] * D[c % M]);
            }
            for (int e = tid; e < K * n; e += nt) {
                const int bb = e / n, r = e - bb * n;
                bv[bb * n0 + r] = Vs[(size_t)r * n + (bb * M + NQ)];
                xv[bb * n0 + r] = 0.0;
                rv[bb * n0 + r] = bv[bb * n0 + r];
            }
            for (int r = tid; r < n; r += nt) {
                perm[r] = r;
                for (int c = n; c < ld; ++c) A[(size_t)r * ld + c] = 0.0f;
            }
            __syncthreads();
            // In-place Gauss-Jordan inversion with partial pivoting (rows swapped
            // in place, perm[] tracks them): afterwards A holds W with
            // W (P r) = (1 - V D)^-1 r, (P r)_k = r_perm[k].
            for (int k = 0; k < n; ++k) {
                if (warp == 0) {
                    float best = -1.0f;
                    int bi = k;
                    for (int r = k + lane; r < n; r += 32) {
                        const float v = fabsf(A[(size_t)r * ld + k]);
                        if (v > best) { best = v; bi = r; }
                    }
                    for (int o = 16; o > 0; o >>= 1) {
                        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
                        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
                    }
                    if (lane == 0) {
                        reinterpret_cast<int *>(red)[0] = bi;
                        reinterpret_cast<float *>(red)[1] = A[(size_t)bi * ld + k];  // the pivot
                    }
                }
                __syncthreads();
                const int pr = reinterpret_cast<int *>(red)[0];
                const float rinv = 1.0f / reinterpret_cast<float *>(red)[1];
                if (pr != k) {
                    for (int c = tid; c < n; c += nt) {
                        const float t = A[(size_t)k * ld + c];
                        A[(size_t)k * ld + c] = A[(size_t)pr * ld + c];
                        A[(size_t)pr * ld + c] = t;
                    }
                    if (tid == 0) {
                        const int t = perm[k];
                        perm[k] = perm[pr];
                        perm[pr] = t;
                    }
                    __syncthreads();
                }
                // the other rows' column-k entries, then row k divided by the pivot
                for (int r = tid; r < n; r += nt) yv[r] = r == k ? 0.0f : A[(size_t)r * ld + k];
                for (int c = tid; c < n; c += nt) A[(size_t)k * ld + c] = c == k ? rinv : A[(size_t)k * ld + c] * rinv;
                __syncthreads();
                // eliminate column k from every other row (one warp per row); the
                // column-k entry becomes -f / pivot (the in-place inverse column)
                // (four columns per lane: the padding columns n..ld-1 stay finite and unused)
                const float4 *Ak4 = reinterpret_cast<const float4 *>(A + (size_t)k * ld);
                for (int r = warp; r < n; r += nw) {
                    if (r == k) continue;
                    const float f = yv[r];
                    float4 *Ar4 = reinterpret_cast<float4 *>(A + (size_t)r * ld);
                    for (int c = lane; c < (ld >> 2); c += 32) {
                        const float4 a = Ar4[c], b = Ak4[c];
                        Ar4[c] = make_float4(fmaf(-f, b.x, a.x), fmaf(-f, b.y, a.y), fmaf(-f, b.z, a.z), fmaf(-f, b.w, a.w));
                    }
                    __syncwarp();  // the lane that updated column k has written it
                    if (lane == 0) A[(size_t)r * ld + k] = -f * A[(size_t)k * ld + k];
                }
                __syncthreads();
            }
            // iterative refinement: y = W (P r) in FP32, x += y, r = b - (x - V D x) in FP64
            bool conv = false;
            int it = 0;
            double ym_prev = 0.0;
            for (; it < kMiMaxRefine && !conv; ++it) {
                double ym = 0.0, xm = 0.0;  // NaN-propagating maxima: a NaN never passes as converged
                for (int r = warp; r < n; r += nw)
                    for (int bb = 0; bb < K; ++bb) {
                        float acc = 0.0f;
                        for (int c = lane; c < n; c += 32)
                            acc = fmaf(A[(size_t)r * ld + c], (float)rv[bb * n0 + perm[c]], acc);
                        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                        if (lane == 0) {
                            const double y = (double)acc, xn = xv[bb * n0 + r] + y;
                            xv[bb * n0 + r] = xn;
                            const double ay = fabs(y), ax = fabs(xn);
                            ym = (ay > ym || ay != ay) ? ay : ym;
                            xm = (ax > xm || ax != ax) ? ax : xm;
                        }
                    }
                ym = mi_block_max(ym, red);
                xm = mi_block_max(xm, red + 32);
                // done when the correction is negligible, or when it has stopped
                // shrinking at the accuracy floor of the FP64 residual (about
                // cond(A) u_64, the accuracy of an FP64 factorisation too)
                conv = ym <= 1e-14 * xm || (it > 0 && ym > 0.25 * ym_prev && ym <= 1e-9 * xm);
                ym_prev = ym;
                if (conv) break;  // (uniform: conv comes from CTA-wide maxima)
                // r = b - x + V (D x): one warp per row, lanes over the columns
                for (int r = warp; r < n; r += nw)
                    for (int bb = 0; bb < K; ++bb) {
                        double acc = 0.0;
                        const double *Vr = Vs + (size_t)r * n;
                        double acc2 = 0.0;  // two chains keep two loads in flight
                        int c = lane;
                        for (; c + 32 < n; c += 64) {
                            const int c1 = c + 32;
                            acc = fma(Vr[c] * D[c < M ? c : c - M], xv[bb * n0 + c], acc);
                            acc2 = fma(Vr[c1] * D[c1 < M ? c1 : c1 - M], xv[bb * n0 + c1], acc2);
                        }
                        if (c < n) acc = fma(Vr[c] * D[c < M ? c : c - M], xv[bb * n0 + c], acc);
                        acc += acc2;
                        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                        if (lane == 0) rv[bb * n0 + r] = bv[bb * n0 + r] - xv[bb * n0 + r] + acc;
                    }
                __syncthreads();
            }
            int steps = conv ? it + 1 : it;  // the loop left by break on convergence
            if (!conv) {
                // The FP32 inverse is too inexact for refinement to converge
                // (cond(A) u_32 ~ 1): solve this system by FP64 Gauss-Jordan
                // elimination with partial pivoting in the slot's second FP64
                // matrix (global memory; rare, so plain), right-hand sides
                // carried along.
                double *G = Vs + (size_t)n0 * n0;
                for (int e = tid; e < n * n; e += nt) {
                    const int r = e / n, c = e - r * n;
                    G[e] = (r == c ? 1.0 : 0.0) - Vs[e] * D[c < M ? c : c - M];
                }
                for (int e = tid; e < K * n; e += nt) xv[(e / n) * n0 + e % n] = bv[(e / n) * n0 + e % n];
                __syncthreads();
                bool ok = true;
                for (int k = 0; k < n; ++k) {
                    if (warp == 0) {
                        double best = -1.0;
                        int bi = k;
                        for (int r = k + lane; r < n; r += 32) {
                            const double v = fabs(G[(size_t)r * n + k]);
                            if (v > best) { best = v; bi = r; }
                        }
                        for (int o = 16; o > 0; o >>= 1) {
                            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
                        }
                        if (lane == 0) reinterpret_cast<int *>(red)[0] = bi;
                    }
                    __syncthreads();
                    const int pr = reinterpret_cast<int *>(red)[0];
                    if (pr != k) {
                        for (int c = tid; c < n; c += nt) {
                            const double t = G[(size_t)k * n + c];
                            G[(size_t)k * n + c] = G[(size_t)pr * n + c];
                            G[(size_t)pr * n + c] = t;
                        }
                        if (tid < K) {
                            const double t = xv[tid * n0 + k];
                            xv[tid * n0 + k] = xv[tid * n0 + pr];
                            xv[tid * n0 + pr] = t;
                        }
                    }
                    __syncthreads();
                    const double piv = G[(size_t)k * n + k];
                    if (piv == 0.0) ok = false;
                    const double rinv = piv != 0.0 ? 1.0 / piv : 0.0;
                    __syncthreads();  // every thread holds the pivot before row k is rescaled
                    for (int c = tid; c < n; c += nt) G[(size_t)k * n + c] *= rinv;
                    if (tid < K) xv[tid * n0 + k] *= rinv;
                    __syncthreads();
                    for (int r = warp; r < n; r += nw) {
                        if (r == k) continue;
                        const double f = G[(size_t)r * n + k];
                        __syncwarp();
                        for (int c = lane; c < n; c += 32) G[(size_t)r * n + c] -= f * G[(size_t)k * n + c];
                        if (lane < K) xv[lane * n0 + r] -= f * xv[lane * n0 + k];
                    }
                    __syncthreads();
                }
                if (ok) {
                    conv = true;
                    steps = kMiMaxRefine + 1;  // marks the FP64 fallback in the status
                }
            }
            if (!conv) worst = -1;
            else if (worst >= 0 && steps > worst) worst = steps;
            if (tid == 0) {
                // on-shell K, T = (1 + i pi mu p K)^-1 K, phases
                double Km[4] = {0, 0, 0, 0};
                for (int a = 0; a < K; ++a)
                    for (int bb = 0; bb < K; ++bb) Km[a * 2 + bb] = xv[bb * n0 + a * M + NQ];
                const double g = kPi * kMu * p;
                double T[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                if (K == 1) {
                    const double dre = 1.0, dim = g * Km[0], dd = dre * dre + dim * dim;
                    T[0] = Km[0] * dre / dd;
                    T[1] = -Km[0] * dim / dd;
                } else {
                    // M = 1 + i g K (complex 2 x 2); T = M^-1 K
                    const double m00r = 1.0, m00i = g * Km[0], m01i = g * Km[1], m10i = g * Km[2], m11r = 1.0,
                                 m11i = g * Km[3];
                    // det = m00 m11 - m01 m10
                    const double detr = m00r * m11r - m00i * m11i + m01i * m10i;
                    const double deti = m00r * m11i + m00i * m11r;
                    const double dd = detr * detr + deti * deti;
                    // inverse = [[m11, -m01], [-m10, m00]] / det
                    const double ir = detr / dd, ii = -deti / dd;
                    const double inv[8] = {m11r * ir - m11i * ii, m11r * ii + m11i * ir,  // (0,0)
                                           m01i * ii, -m01i * ir,                          // (0,1) = -i m01i / det
                                           m10i * ii, -m10i * ir,                          // (1,0)
                                           m00r * ir - m00i * ii, m00r * ii + m00i * ir};  // (1,1)
                    for (int a = 0; a < 2; ++a)
                        for (int bb = 0; bb < 2; ++bb) {
                            double re = 0.0, im = 0.0;
                            for (int k = 0; k < 2; ++k) {
                                re += inv[(a * 2 + k) * 2] * Km[k * 2 + bb];
                                im += inv[(a * 2 + k) * 2 + 1] * Km[k * 2 + bb];
                            }
                            T[(a * 2 + bb) * 2] = re;
                            T[(a * 2 + bb) * 2 + 1] = im;
                        }
                }
                const size_t o = ((size_t)smp * n_ch_total + cidx) * n_I + ie;
                phases_of_T(K, p, T, ph + o * 3);
                if (k_out)
                    for (int k = 0; k < 4; ++k) k_out[o * 4 + k] = Km[k];
            }
            __syncthreads();
        }
        if (tid == 0) {
            status[(size_t)smp * n_ch_total + cidx] = worst;
            if (worst < 0) record_error(err, kDevNoConverge);
        }
    }
}

cudaError_t launch_mi_solve(const MiChanDev *chans_dev, const int *work_dev, int n_work, int n, int n_ch_total,
                            int n_samples, int NQ, const double *kg, const double *wg, int n_terms,
                            const double *coeffs, const double *Vg, const double *Von, int n_I, const double *e_int,
                            double *Vs, int slots, double *ph, double *k_out, int *status, int *err,
                            cudaStream_t st)
{
    const size_t smem = mi_smem(n, NQ + 1);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    raise_smem_limit((const void *)k_mi_solve, smem);
    k_mi_solve<<<slots, kMiThreads, smem, counted(st)>>>(chans_dev, work_dev, n_work, n_ch_total, n_samples, NQ, kg, wg, n_terms,
                                                coeffs, Vg, Von, n_I, e_int, Vs, ph, k_out, status, err);
    return cudaGetLastError();
}

int mi_slots_per_sm(int n, int NQ)
{
    const size_t smem = mi_smem(n, NQ + 1);
    raise_smem_limit((const void *)k_mi_solve, smem);
    int blocks = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_mi_solve, kMiThreads, smem);
    return blocks;
}

// ------------------------------------------------------------------------------------- observables
// Phases at the requested energies by linear interpolation in T_lab between
// consecutive interpolation energies (end segments extended, delta unwrapped
// by multiples of 180 deg), and the np total cross section.  One thread per
// (sample, energy).
__global__ void k_mi_observables(const MiChanDev *chans, int n_ch, int n_samples, int n_I, const double *e_int,
                                 const double *ph, int n_E, const double *e_lab, double *delta, double *sigma)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n_samples * n_E) return;
    const int e = (int)(idx % n_E), smp = (int)(idx / n_E);
    const double E = e_lab[e], p = sqrt(kMn * E / 2.0) / kHbarc, rad = kPi / 180.0;
    int lo = -1, hi = n_I - 1;  // largest j with e_int[j] <= E
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (e_int[mid] <= E) lo = mid;
        else hi = mid - 1;
    }
    const int j = lo < 0 ? 0 : (lo > n_I - 2 ? n_I - 2 : lo);
    const double w = (E - e_int[j]) / (e_int[j + 1] - e_int[j]);
    double acc = 0.0;
    for (int c = 0; c < n_ch; ++c) {
        const MiChanDev ch = chans[c];
        const double *pc = ph + ((size_t)smp * n_ch + c) * n_I * 3;
        double out[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < ch.K; ++k) {
            const double d0 = pc[3 * j + k];
            double d1 = pc[3 * (j + 1) + k];
            d1 += 180.0 * round((d0 - d1) / 180.0);
            double d = d0 + w * (d1 - d0);
            if (isfinite(d)) {
                while (d > 90.0) d -= 180.0;
                while (d <= -90.0) d += 180.0;
            }
            out[k] = d;
        }
        if (ch.K == 2) out[2] = pc[3 * j + 2] + w * (pc[3 * (j + 1) + 2] - pc[3 * j + 2]);
        if (delta) {
            double *d = delta + (((size_t)smp * n_ch + c) * n_E + e) * 3;
            d[0] = out[0];
            d[1] = out[1];
            d[2] = out[2];
        }
        if (ch.tz == 0) {
            if (ch.K == 1) {
                acc += (2.0 * ch.J + 1.0) * (1.0 - cos(2.0 * out[0] * rad));
            } else {
                const double c2e = cos(2.0 * out[2] * rad);
                acc += (2.0 * ch.J + 1.0) *
                       ((1.0 - c2e * cos(2.0 * out[0] * rad)) + (1.0 - c2e * cos(2.0 * out[1] * rad)));
            }
        }
    }
    if (sigma) sigma[idx] = kPi / (2.0 * p * p) * 10.0 * acc;
}

cudaError_t launch_mi_observables(const MiChanDev *chans_dev, int n_ch, int n_samples, int n_I, const double *e_int,
                                  const double *ph, int n_E, const double *e_lab, double *delta, double *sigma,
                                  cudaStream_t st)
{
    const size_t total = (size_t)n_samples * n_E;
    k_mi_observables<<<(unsigned)((total + 127) / 128), 128, 0, counted(st)>>>(chans_dev, n_ch, n_samples, n_I, e_int, ph, n_E,
                                                                       e_lab, delta, sigma);
    return cudaGetLastError();
}

}  // namespace wpcd
