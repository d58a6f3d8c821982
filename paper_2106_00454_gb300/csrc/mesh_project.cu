// mesh_project.cu -- (a0) free-wave-packet mesh and (a1) projection of the
// potential terms onto the wave-packet basis (Sec. 3.2 step 1 and Eq. "WP
// potential matrix identity").  FP64 on the CUDA cores.
#include <math.h>

#include "potential.cuh"
#include "wpcd_internal.cuh"

namespace wpcd {

// ---------------------------------------------------------------------------------------------
// Gauss-Legendre rule on [-1, 1]: one thread per node pair, Newton iteration on
// P_n from the three-term recurrence.
// ---------------------------------------------------------------------------------------------
__global__ void k_gauss_legendre(int n, double *x, double *w)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int m = (n + 1) / 2;
    if (i >= m) return;
    double z = cos(kPi * (i + 0.75) / (n + 0.5));
    double pcur = z, pm1 = 1.0, dp = 1.0;
    for (int it = 0; it < 100; ++it) {
        pm1 = 1.0;
        pcur = z;
        for (int j = 2; j <= n; ++j) {
            double pn = ((2.0 * j - 1.0) * z * pcur - (j - 1.0) * pm1) / j;
            pm1 = pcur;
            pcur = pn;
        }
        dp = n * (z * pcur - pm1) / (z * z - 1.0);
        double dz = pcur / dp;
        z -= dz;
        if (fabs(dz) < 1e-16) break;
    }
    pm1 = 1.0;
    pcur = z;
    for (int j = 2; j <= n; ++j) {
        double pn = ((2.0 * j - 1.0) * z * pcur - (j - 1.0) * pm1) / j;
        pm1 = pcur;
        pcur = pn;
    }
    dp = n * (z * pcur - pm1) / (z * z - 1.0);
    double wi = 2.0 / ((1.0 - z * z) * dp * dp);
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = wi;
    w[n - 1 - i] = wi;
    if ((n & 1) && i == m - 1) x[i] = 0.0;
}

cudaError_t launch_gauss_legendre(int n, double *x, double *w, cudaStream_t st)
{
    int m = (n + 1) / 2;
    k_gauss_legendre<<<(m + 63) / 64, 64, 0, counted(st)>>>(n, x, w);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Mesh: N+1 boundaries, Q-point rule per bin, and the exact diagonal of h0 in the
// packet basis, <x_i|h0|x_i> = (1/N_i) int_{D_i} dk f(k)^2 k^2/(2 mu).
// One block; thread j handles boundary j and bin j.
// ---------------------------------------------------------------------------------------------
__global__ void k_mesh(int N, int kind, double alpha, double t, double kmax, int Q, int wp_kind, const double *glx,
                       const double *glw, double *kb, double *kq, double *wq, double *h0)
{
    extern __shared__ double sk[];  // N+1
    for (int j = threadIdx.x; j <= N; j += blockDim.x) {
        double v;
        if (j == 0) {
            v = 0.0;
        } else if (kind == 0) {
            double thmax = atan(pow(kmax / alpha, 1.0 / t));
            v = (j == N) ? kmax : alpha * pow(tan(j * thmax / N), t);
        } else {
            v = alpha * pow(tan((2.0 * j - 1.0) * kPi / (4.0 * N)), t);
        }
        sk[j] = v;
        kb[j] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double a = sk[i], b = sk[i + 1];
        for (int q = 0; q < Q; ++q) {
            kq[i * Q + q] = 0.5 * (a + b) + 0.5 * (b - a) * glx[q];
            wq[i * Q + q] = 0.5 * (b - a) * glw[q];
        }
        if (wp_kind == 0) {
            h0[i] = (b * b * b - a * a * a) / (3.0 * (b - a)) / (2.0 * kMu);
        } else {
            h0[i] = 0.5 * (a * a + b * b) / (2.0 * kMu);
        }
    }
}

cudaError_t launch_mesh(int N, int kind, double alpha, double t, double kmax, int Q, int wp_kind,
                        const double *glx, const double *glw, double *kb, double *kq, double *wq, double *h0,
                        cudaStream_t st)
{
    k_mesh<<<1, 256, (N + 1) * sizeof(double), counted(st)>>>(N, kind, alpha, t, kmax, Q, wp_kind, glx, glw, kb, kq, wq, h0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Projection.  Every CTA owns one pair of bins (i <= j) of one mesh and all the
// channels that use that mesh; each thread one fine pair (a in D_i, b in D_j).
// It evaluates v_t(k_a, k_b) for every term, multiplies by
//   omega_a omega_b,  omega_a = w_a k_a f(k_a) / sqrt(N_i),
// and the CTA sums over its Q x Q pairs.  The matrix element and its mirror
// V[(b,j),(a,i)] = V[(a,i),(b,j)] are written together (v^{l'l}(p',p) =
// v^{ll'}(p,p')).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double wp_f(int wp_kind, double k) { return wp_kind == 0 ? 1.0 : sqrt(k / kMu); }
__device__ __forceinline__ double wp_norm(int wp_kind, double a, double b)
{
    return wp_kind == 0 ? (b - a) : (b * b - a * a) / (2.0 * kMu);
}

// Sum over the CTA (blockDim <= 1024, multiple of 32).  Every thread gets the total.
__device__ __forceinline__ double cta_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double tot = 0.0;
    for (int k = 0; k < nw; ++k) tot += red[k];
    return tot;
}

// Ibuf (Yukawa only, may be NULL): the angle integrals of every fine pair,
// [pair][mass][16] FP32 from the tensor-core contraction (project_tc.cu), used
// instead of the FP64 angle sums.
template <int GEN>
__global__ void __launch_bounds__(256) k_project(const ChanDev *chans, const int *group, int n_group, int N, int Q,
                                                 int Lmax, const double *gp, const double *angx, const double *angw,
                                                 int n_terms, const float *Ibuf)
{
    // decode the bin pair (i <= j) from the linear block index over the upper triangle
    int b = blockIdx.x;
    int j = (int)((sqrt(8.0 * b + 1.0) - 1.0) * 0.5);
    while ((j + 1) * (j + 2) / 2 <= b) ++j;
    while (j * (j + 1) / 2 > b) --j;
    int i = b - j * (j + 1) / 2;
    if (j >= N) return;

    __shared__ double wpl[kAngleQ][kLmaxReg + 1];  // w_x P_L(x)
    __shared__ double ax[kAngleQ];
    __shared__ double red[8];
    const int Lm = (Lmax < kLmaxReg) ? Lmax : kLmaxReg;
    if (GEN == WPCD_GEN_YUKAWA && !Ibuf) {
        angle_tables(angx, angw, Lm, wpl, ax);
        __syncthreads();
    }

    const ChanDev c0 = chans[group[0]];
    const int qa = threadIdx.x / Q, qb = threadIdx.x % Q;
    const bool live = threadIdx.x < Q * Q;
    const int a = i * Q + (live ? qa : 0), bb = j * Q + (live ? qb : 0);
    const double pp = c0.kq[a], p = c0.kq[bb];
    double om = 0.0;
    if (live) {
        om = c0.wq[a] * pp * wp_f(c0.wp_kind, pp) / sqrt(wp_norm(c0.wp_kind, c0.kb[i], c0.kb[i + 1]));
        om *= c0.wq[bb] * p * wp_f(c0.wp_kind, p) / sqrt(wp_norm(c0.wp_kind, c0.kb[j], c0.kb[j + 1]));
    }

    double I1[kLmaxReg + 1], I2[kLmaxReg + 1], I3[kLmaxReg + 1];
    double R = 0.0;
    if (GEN == WPCD_GEN_YUKAWA) {
        if (Ibuf) {
            const float *Ip = Ibuf + ((size_t)b * Q * Q + (live ? threadIdx.x : 0)) * 48;
#pragma unroll
            for (int L = 0; L <= kLmaxReg; ++L) {
                const bool on = L <= Lm;
                I1[L] = on ? (double)Ip[L] : 0.0;
                I2[L] = on ? (double)Ip[16 + L] : 0.0;
                I3[L] = on ? (double)Ip[32 + L] : 0.0;
            }
            R = exp(-(pp * pp + p * p) / (gp[3] * gp[3]));
        } else {
            yukawa_angle_integrals(gp, wpl, ax, Lm, pp, p, I1, I2, I3, R);
        }
    }

    for (int g = 0; g < n_group; ++g) {
        const int cidx = group[g];
        const ChanDev ch = chans[cidx];
        const int K = ch.K, n = ch.n;
        for (int al = 0; al < K; ++al)
            for (int be = 0; be < K; ++be) {
                const int lp = ch.coupled ? (al == 0 ? ch.J - 1 : ch.J + 1) : ch.l;
                const int l = ch.coupled ? (be == 0 ? ch.J - 1 : ch.J + 1) : ch.l;
                double tv[kMaxTerms];
                potential_terms<GEN>(gp, ch.s, ch.J, ch.tz, lp, l, pp, p, I1, I2, I3, R, tv);
                for (int t = 0; t < n_terms; ++t) {
                    double v = cta_sum(live ? om * tv[t] : 0.0, red);
                    if (threadIdx.x == 0) {
                        double *Vt = const_cast<double *>(ch.V) + (size_t)t * n * n;
                        Vt[(size_t)(al * N + i) * n + (be * N + j)] = v;
                        Vt[(size_t)(be * N + j) * n + (al * N + i)] = v;
                    }
                }
            }
    }
}

static int proj_threads(int Q) { return ((Q * Q + 31) / 32) * 32; }

cudaError_t launch_project_yukawa(const ChanDev *chans_dev, const int *group_dev, int n_group, int N, int Q, int Lmax,
                                  const double *gp_dev, const double *angx, const double *angw, int n_terms,
                                  cudaStream_t st, const float *Ibuf)
{
    int nblk = N * (N + 1) / 2;
    k_project<WPCD_GEN_YUKAWA><<<nblk, proj_threads(Q), 0, counted(st)>>>(chans_dev, group_dev, n_group, N, Q, Lmax, gp_dev,
                                                                 angx, angw, n_terms, Ibuf);
    return cudaGetLastError();
}

// Yamaguchi parameters travel in the same device parameter buffer as the Yukawa set.
cudaError_t launch_project_yamaguchi_gp(const ChanDev *chans_dev, const int *group_dev, int n_group, int N, int Q,
                                        const double *gp_dev, cudaStream_t st)
{
    int nblk = N * (N + 1) / 2;
    k_project<WPCD_GEN_YAMAGUCHI><<<nblk, proj_threads(Q), 0, counted(st)>>>(chans_dev, group_dev, n_group, N, Q, 0, gp_dev,
                                                                    nullptr, nullptr, 1, nullptr);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Caller-supplied fine-grid values: the same bin reduction, over all (i, j) and
// l-blocks of one channel.  vfine: [n_terms][K*NQ][K*NQ].
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_project_fine(const ChanDev *chans, int c, const double *vfine, int n_terms)
{
    const ChanDev ch = chans[c];
    const int N = ch.N, Q = ch.Q, K = ch.K, n = ch.n, NQ = N * Q;
    const int i = blockIdx.x, j = blockIdx.y;
    __shared__ double red[8];
    const int qa = threadIdx.x / Q, qb = threadIdx.x % Q;
    const bool live = threadIdx.x < Q * Q;
    const int a = i * Q + (live ? qa : 0), b = j * Q + (live ? qb : 0);
    double om = 0.0;
    if (live) {
        om = ch.wq[a] * ch.kq[a] * wp_f(ch.wp_kind, ch.kq[a]) / sqrt(wp_norm(ch.wp_kind, ch.kb[i], ch.kb[i + 1]));
        om *= ch.wq[b] * ch.kq[b] * wp_f(ch.wp_kind, ch.kq[b]) / sqrt(wp_norm(ch.wp_kind, ch.kb[j], ch.kb[j + 1]));
    }
    const size_t KNQ = (size_t)K * NQ;
    for (int t = 0; t < n_terms; ++t)
        for (int al = 0; al < K; ++al)
            for (int be = 0; be < K; ++be) {
                double v = 0.0;
                if (live) v = om * vfine[(size_t)t * KNQ * KNQ + (size_t)(al * NQ + a) * KNQ + (be * NQ + b)];
                v = cta_sum(v, red);
                if (threadIdx.x == 0) {
                    double *Vt = const_cast<double *>(ch.V) + (size_t)t * n * n;
                    Vt[(size_t)(al * N + i) * n + (be * N + j)] = v;
                }
            }
}

cudaError_t launch_project_fine(const ChanDev *chans_dev, int c, const ChanDev &ch_host, const double *vfine,
                                int n_terms, cudaStream_t st)
{
    dim3 grid(ch_host.N, ch_host.N);
    k_project_fine<<<grid, proj_threads(ch_host.Q), 0, counted(st)>>>(chans_dev, c, vfine, n_terms);
    return cudaGetLastError();
}

}  // namespace wpcd
