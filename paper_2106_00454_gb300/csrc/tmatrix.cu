// tmatrix.cu -- (a4) SWP boundaries, (a5) energy-averaged resolvent, (a6) VC
// rows and on-shell T, (a7) continuum T, S and phase shifts at the bin
// midpoints, (a8) interpolation to the requested energies and the np total
// cross section.  FP64 throughout (the logarithms of the resolvent and the
// phase extraction need it even on the reduced-precision path).
#include <math.h>

#include "wpcd_internal.cuh"

namespace wpcd {

constexpr int kTThreads = 256;

// ---------------------------------------------------------------------------------------------
// Energy plan: per channel and energy, the free bin holding p(E) and the
// midpoint segment used for interpolation; per channel, the distinct bins
// whose T is needed (the bin itself and both ends of its segment).
// ---------------------------------------------------------------------------------------------
__global__ void k_plan(const ChanDev *chans, int n_ch, int maxN, const double *e_lab, int n_E, PlanDev plan, int *err)
{
    const int c = blockIdx.x, ps = blockIdx.y;
    const ChanDev ch = chans[c];
    const int N = ch.N;
    const int nE = plan_nE(plan, ps, n_E);
    const size_t pc = (size_t)ps * n_ch + c;
    __shared__ int mark[kMaxNwp];
    for (int i = threadIdx.x; i < N; i += blockDim.x) mark[i] = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < nE; e += blockDim.x) {
        const double T = e_lab[(size_t)ps * n_E + e];
        const double p = sqrt(kMn * T / 2.0) / kHbarc;
        if (c == 0) plan.pE[(size_t)ps * n_E + e] = p;
        int bin = 0, j = 0;
        if (!(T > 0.0) || !(p < ch.kb[N])) {
            record_error(err, kDevEnergyOutside);
        } else {
            int lo = 0, hi = N - 1;  // largest i with kb[i] <= p
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (ch.kb[mid] <= p) lo = mid;
                else hi = mid - 1;
            }
            bin = lo;
            lo = -1;
            hi = N - 1;  // largest j with kbar_j <= p (or -1)
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (0.5 * (ch.kb[mid] + ch.kb[mid + 1]) <= p) lo = mid;
                else hi = mid - 1;
            }
            j = lo < 0 ? 0 : (lo > N - 2 ? N - 2 : lo);
        }
        plan.bin[pc * n_E + e] = bin;
        plan.brk[pc * n_E + e] = j;
        atomicExch(&mark[bin], 1);
        atomicExch(&mark[j], 1);
        atomicExch(&mark[j + 1], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int cnt = 0;
        for (int i = 0; i < N; ++i)
            if (mark[i]) plan.list[pc * maxN + cnt++] = i;
        plan.cnt[pc] = cnt;
    }
}

cudaError_t launch_plan(const ChanDev *chans_dev, int n_ch, int maxN, const double *e_lab, int n_E, PlanDev plan,
                        int *err, cudaStream_t st, int n_plans)
{
    k_plan<<<dim3(n_ch, n_plans), 256, 0, st>>>(chans_dev, n_ch, maxN, e_lab, n_E, plan, err);
    return cudaGetLastError();
}

__device__ __forceinline__ double xlogabs(double d) { return d == 0.0 ? 0.0 : d * log(fabs(d)); }

template <int NV>
__device__ __forceinline__ void block_sum_vec(double *v, double *red /* [NV][32] */)
{
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) red[k * 32 + w] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double t = 0.0;
        for (int q = 0; q < nw; ++q) t += red[k * 32 + q];
        v[k] = t;
    }
}

// ---------------------------------------------------------------------------------------------
// T at the needed bins.  One CTA per (sample, channel).
//  - SWP boundaries (Eq. "pseudostate wave packet boundaries"): the positive
//    eigenvalues of each branch give B_1 = 0, B_i = (e_{i-1}+e_i)/2,
//    B_{m+1} = e_m + (B_m - B_{m-1})/2.  Coupled channels: the positive
//    eigenvalues, sorted, are dealt to the two branches alternately from the
//    top (largest -> branch 1).
//  - for each needed free bin i: the rows (a, i) of V (rebuilt from the terms
//    and the sample's coefficients), R = V_rows C, the resolvent averaged
//    over the free bin [E_i, E_{i+1}]
//      gbar_s = [X(Eb,B_s) - X(Ea,B_s) - X(Eb,B_s+1) + X(Ea,B_s+1)]/(dE dB)
//               - i pi |[Ea,Eb] ^ [B_s,B_s+1]| / (dE dB),   X(a,b) = (a-b) ln|a-b|,
//    or ln((Eb - e_b)/(Ea - e_b))/dE for a bound state e_b < 0, and
//      T_ab = V_(a,i),(b,i) + sum_s R_as gbar_s R_bs.
//  - continuum T at q = the bin midpoint: T f(q)^2 / (N_i q^2); S = 1 - 2 pi i
//    mu q T; phases (Stapp for coupled channels).
// tbin: [S][n_ch][maxN][K][K] complex (8 doubles per bin); phbin: [S][n_ch][maxN][3].
// ---------------------------------------------------------------------------------------------
// TC: eigenvector type (double on the FP64 path; float on the mixed path, where
// the VC rows are accumulated in FP32 and everything after them stays FP64).
template <typename TC>
__global__ void __launch_bounds__(kTThreads) k_tbin(const ChanDev *chans, int n_ch, int n_terms, const double *coeffs,
                                                    const double *eps_all, const TC *C_all, PlanDev plan, int maxN,
                                                    double *tbin, double *phbin, int *err)
{
    const int c = blockIdx.x % n_ch, smp = blockIdx.x / n_ch;
    const ChanDev ch = chans[c];
    const int n = ch.n, N = ch.N, K = ch.K;
    const int tid = threadIdx.x, nt = blockDim.x;
    if ((size_t)dyn_smem_bytes() < tbin_smem_doubles(n) * sizeof(double)) {  // launch/layout mismatch
        if (tid == 0) record_error(err, kDevBadSize);
        return;
    }
    extern __shared__ double sm[];
    double *eps = sm;              // n
    double *Eb = eps + n;          // 2 x n   branch members
    double *Bb = Eb + 2 * n;       // 2 x (n+1) branch boundaries
    double *lo = Bb + 2 * (n + 1); // n  lower SWP boundary of eigenvalue s
    double *hi = lo + n;           // n  upper
    double *vrow = hi + n;         // K x n
    double *R = vrow + 2 * n;      // K x n
    double *red = R + 2 * n;       // 6 x 32
    __shared__ int s_nb, s_bad;

    const double *eg = eps_all + ch.eps_off + (size_t)smp * n;
    const TC *C = C_all + ch.c_off + (size_t)smp * n * n;
    TC *vrowc = reinterpret_cast<TC *>(red + 6 * 32);  // K x n copy of the V rows in the accumulation type
    const double *cf = coeffs ? coeffs + (size_t)smp * (n_terms - 1) : nullptr;

    if (tid == 0) { s_nb = 0; s_bad = 0; }
    for (int s = tid; s < n; s += nt) eps[s] = eg[s];
    __syncthreads();
    for (int s = tid; s < n; s += nt)
        if (eps[s] < 0.0 && (s == n - 1 || !(eps[s + 1] < 0.0))) s_nb = s + 1;
    __syncthreads();
    const int nb = s_nb, P = n - nb;
    int mcount[2];
    mcount[0] = (K == 2) ? P / 2 : P;
    mcount[1] = (K == 2) ? (P + 1) / 2 : 0;
    // branch members, ascending within each branch
    for (int s = nb + tid; s < n; s += nt) {
        const int d = s - nb;
        const int b = (K == 2) ? (((n - 1 - s) & 1) == 0 ? 1 : 0) : 0;
        const int pos = (K == 2) ? d / 2 : d;
        Eb[b * n + pos] = eps[s];
    }
    __syncthreads();
    for (int b = 0; b < K; ++b) {
        const int m = mcount[b];
        if (m < 2) {
            if (tid == 0) s_bad = 1;
            continue;
        }
        double *B = Bb + b * (n + 1);
        const double *E = Eb + b * n;
        for (int i = tid; i < m; i += nt) B[i] = (i == 0) ? 0.0 : 0.5 * (E[i - 1] + E[i]);
    }
    __syncthreads();
    if (s_bad) {
        if (tid == 0) record_error(err, kDevBranch);
        return;
    }
    if (tid < K) {
        const int m = mcount[tid];
        double *B = Bb + tid * (n + 1);
        B[m] = Eb[tid * n + m - 1] + 0.5 * (B[m - 1] - B[m - 2]);
    }
    __syncthreads();
    for (int s = nb + tid; s < n; s += nt) {
        const int d = s - nb;
        const int b = (K == 2) ? (((n - 1 - s) & 1) == 0 ? 1 : 0) : 0;
        const int pos = (K == 2) ? d / 2 : d;
        lo[s] = Bb[b * (n + 1) + pos];
        hi[s] = Bb[b * (n + 1) + pos + 1];
    }
    __syncthreads();

    const size_t pc = (size_t)plan_of(plan, smp) * n_ch + c;
    const int cnt = plan.cnt[pc];
    const size_t obase = ((size_t)smp * n_ch + c) * maxN;
    for (int ii = 0; ii < cnt; ++ii) {
        const int i = plan.list[pc * maxN + ii];
        // rows (a, i) of V = V0 + sum_a c_a V_a
        for (int e = tid; e < K * n; e += nt) {
            const int a = e / n, jj = e - a * n;
            const size_t off = (size_t)(a * N + i) * n + jj;
            double v = ch.V[off];
            for (int t = 1; t < n_terms; ++t) v = fma(cf[t - 1], ch.V[(size_t)t * n * n + off], v);
            vrow[a * n + jj] = v;
            vrowc[a * n + jj] = (TC)v;
        }
        __syncthreads();
        // R = V_rows C
        for (int e = tid; e < K * n; e += nt) {
            const int a = e / n, s = e - a * n;
            const TC *vr = vrowc + a * n;
            TC acc = 0;
            for (int j = 0; j < n; ++j) acc = fma(vr[j], C[(size_t)j * n + s], acc);
            R[a * n + s] = (double)acc;
        }
        __syncthreads();
        const double Ea = ch.kb[i] * ch.kb[i] / (2.0 * kMu), Ebn = ch.kb[i + 1] * ch.kb[i + 1] / (2.0 * kMu);
        const double dE = Ebn - Ea;
        // D(B) = X(Eb, B) - X(Ea, B) once per SWP boundary of each branch (the
        // branch-member array is free by now); state s then needs D(B_s) - D(B_s+1)
        const int dstride = (K == 2) ? (n >> 1) + 2 : n + 1;
        double *Dv = Eb;
        for (int e = tid; e < K * dstride; e += nt) {
            const int b = e / dstride, pos = e - b * dstride;
            if (pos <= mcount[b]) {
                const double B = Bb[b * (n + 1) + pos];
                Dv[e] = xlogabs(Ebn - B) - xlogabs(Ea - B);
            }
        }
        __syncthreads();
        double acc[6] = {0, 0, 0, 0, 0, 0};  // (00 re, im), (01 re, im), (11 re, im)
        for (int s = tid; s < n; s += nt) {
            double gre, gim;
            if (s < nb) {
                gre = log((Ebn - eps[s]) / (Ea - eps[s])) / dE;
                gim = 0.0;
            } else {
                const double b0 = lo[s], b1 = hi[s], dB = b1 - b0;
                const int d = s - nb;
                const int b = (K == 2) ? (((n - 1 - s) & 1) == 0 ? 1 : 0) : 0;
                const int pos = (K == 2) ? d / 2 : d;
                const double num = Dv[b * dstride + pos] - Dv[b * dstride + pos + 1];
                gre = num / (dE * dB);
                const double l = Ea > b0 ? Ea : b0, h = Ebn < b1 ? Ebn : b1;
                gim = (h > l) ? -kPi * (h - l) / (dE * dB) : 0.0;
            }
            const double r0 = R[s];
            acc[0] = fma(r0 * r0, gre, acc[0]);
            acc[1] = fma(r0 * r0, gim, acc[1]);
            if (K == 2) {
                const double r1 = R[n + s];
                acc[2] = fma(r0 * r1, gre, acc[2]);
                acc[3] = fma(r0 * r1, gim, acc[3]);
                acc[4] = fma(r1 * r1, gre, acc[4]);
                acc[5] = fma(r1 * r1, gim, acc[5]);
            }
        }
        block_sum_vec<6>(acc, red);
        if (tid == 0) {
            const double kbar = 0.5 * (ch.kb[i] + ch.kb[i + 1]);
            const double Ni = ch.wp_kind == 0 ? (ch.kb[i + 1] - ch.kb[i]) : dE;
            const double f2 = ch.wp_kind == 0 ? 1.0 : kbar / kMu;
            const double fac = f2 / (Ni * kbar * kbar);
            double T[8];  // complex 2x2, row-major
            T[0] = fac * (vrow[i] + acc[0]);
            T[1] = fac * acc[1];
            if (K == 2) {
                T[2] = fac * (vrow[N + i] + acc[2]);
                T[3] = fac * acc[3];
                T[4] = fac * (vrow[n + i] + acc[2]);
                T[5] = fac * acc[3];
                T[6] = fac * (vrow[n + N + i] + acc[4]);
                T[7] = fac * acc[5];
            } else {
                T[2] = T[3] = T[4] = T[5] = T[6] = T[7] = 0.0;
            }
            double *to = tbin + (obase + i) * 8;
            for (int k = 0; k < 8; ++k) to[k] = T[k];
            // S = 1 - 2 pi i mu q T
            const double g = 2.0 * kPi * kMu * kbar;
            double *po = phbin + (obase + i) * 3;
            const double deg = 180.0 / kPi;
            if (K == 1) {
                const double sre = 1.0 + g * T[1], sim = -g * T[0];
                po[0] = 0.5 * atan2(sim, sre) * deg;
                po[1] = 0.0;
                po[2] = 0.0;
            } else {
                const double s11r = 1.0 + g * T[1], s11i = -g * T[0];
                const double s22r = 1.0 + g * T[7], s22i = -g * T[6];
                const double s12r = g * T[3], s12i = -g * T[2];
                const double dm = 0.5 * atan2(s11i, s11r), dp = 0.5 * atan2(s22i, s22r);
                const double ph = dm + dp;
                double x = s12i * cos(ph) - s12r * sin(ph);  // Re(-i S12 e^{-i ph})
                x = x > 1.0 ? 1.0 : (x < -1.0 ? -1.0 : x);
                po[0] = dm * deg;
                po[1] = dp * deg;
                po[2] = 0.5 * asin(x) * deg;
            }
        }
        __syncthreads();
    }
}

size_t tbin_smem_bytes(int nmax) { return tbin_smem_doubles(nmax) * sizeof(double); }

cudaError_t launch_tbin(const ChanDev *chans_dev, int n_ch, int n_samples, int n_terms, const double *coeffs,
                        const double *eps_all, const double *C_all, PlanDev plan, int maxN, double *tbin,
                        double *phbin, int *err, cudaStream_t st)
{
    const size_t smem = tbin_smem_bytes(2 * maxN);
    cudaFuncSetAttribute(k_tbin<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_tbin<double><<<(unsigned)(n_samples * n_ch), kTThreads, smem, st>>>(chans_dev, n_ch, n_terms, coeffs, eps_all,
                                                                           C_all, plan, maxN, tbin, phbin, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// T at the requested energies: the bin value of the bin holding p(E).
// t_out: [S][n_ch][n_E][2][2] complex.
// ---------------------------------------------------------------------------------------------
__global__ void k_gather_t(int n_ch, int n_samples, int n_E, int maxN, PlanDev plan, const double *tbin, double *t_out)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)n_samples * n_ch * n_E;
    if (idx >= total) return;
    const int e = (int)(idx % n_E);
    const size_t sc = idx / n_E;
    const int c = (int)(sc % n_ch);
    const int ps = plan_of(plan, (int)(sc / n_ch));
    if (e >= plan_nE(plan, ps, n_E)) return;
    const int bin = plan.bin[((size_t)ps * n_ch + c) * n_E + e];
    const double *src = tbin + (sc * maxN + bin) * 8;
    double *dst = t_out + idx * 8;
    const double2 *s2 = reinterpret_cast<const double2 *>(src);
    double2 *d2 = reinterpret_cast<double2 *>(dst);
#pragma unroll
    for (int k = 0; k < 4; ++k) d2[k] = s2[k];
}

cudaError_t launch_gather_t(const ChanDev *chans_dev, int n_ch, int n_samples, int n_E, int maxN, PlanDev plan,
                            const double *tbin, double *t_out, cudaStream_t st)
{
    (void)chans_dev;
    const size_t total = (size_t)n_samples * n_ch * n_E;
    k_gather_t<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(n_ch, n_samples, n_E, maxN, plan, tbin, t_out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Phases interpolated linearly in p between the midpoints of the segment j,
// j+1 (extended past the end midpoints), after moving delta_{j+1} by a
// multiple of 180 deg to within 90 deg of delta_j; result mapped to
// (-90, 90].  Total cross section sigma = pi/(2p^2) sum (2J+1) sum_l Re(1 -
// S_ll) over the np channels (tz = 0), with S rebuilt from the interpolated
// Stapp parameters.  One thread per (sample, energy).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double wrap90(double d)
{
    if (!isfinite(d)) return d;
    while (d > 90.0) d -= 180.0;
    while (d <= -90.0) d += 180.0;
    return d;
}

__global__ void k_observables(const ChanDev *chans, int n_ch, int n_samples, int n_E, int maxN, PlanDev plan,
                              const double *phbin, double *delta, double *sigma)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n_samples * n_E) return;
    const int e = (int)(idx % n_E);
    const int smp = (int)(idx / n_E);
    const int ps = plan_of(plan, smp);
    if (e >= plan_nE(plan, ps, n_E)) return;
    const double p = plan.pE[(size_t)ps * n_E + e];
    const double rad = kPi / 180.0;
    double acc = 0.0;
    for (int c = 0; c < n_ch; ++c) {
        const ChanDev ch = chans[c];
        const int j = plan.brk[((size_t)ps * n_ch + c) * n_E + e];
        const double q0 = 0.5 * (ch.kb[j] + ch.kb[j + 1]), q1 = 0.5 * (ch.kb[j + 1] + ch.kb[j + 2]);
        const double w = (p - q0) / (q1 - q0);
        const double *ph = phbin + (((size_t)smp * n_ch + c) * maxN) * 3;
        double out[3];
        const int ncomp = ch.K == 2 ? 2 : 1;
        for (int k = 0; k < ncomp; ++k) {
            const double d0 = ph[3 * j + k];
            double d1 = ph[3 * (j + 1) + k];
            d1 += 180.0 * round((d0 - d1) / 180.0);
            out[k] = wrap90(d0 + w * (d1 - d0));
        }
        if (ch.K == 2) {
            const double e0 = ph[3 * j + 2], e1 = ph[3 * (j + 1) + 2];
            out[2] = e0 + w * (e1 - e0);
        } else {
            out[1] = 0.0;
            out[2] = 0.0;
        }
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

cudaError_t launch_observables(const ChanDev *chans_dev, int n_ch, int n_samples, int n_E, int maxN, PlanDev plan,
                               const double *phbin, double *delta, double *sigma, cudaStream_t st)
{
    const size_t total = (size_t)n_samples * n_E;
    k_observables<<<(unsigned)((total + 127) / 128), 128, 0, st>>>(chans_dev, n_ch, n_samples, n_E, maxN, plan, phbin,
                                                                    delta, sigma);
    return cudaGetLastError();
}

}  // namespace wpcd
