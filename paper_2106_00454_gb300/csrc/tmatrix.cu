// tmatrix.cu -- (a4) SWP boundaries, (a5) energy-averaged resolvent, (a6) VC
// rows and on-shell T, (a7) continuum T, S and phase shifts at the bin
// midpoints, (a8) interpolation to the requested energies and the np total
// cross section.  FP64 throughout (the logarithms of the resolvent and the
// phase extraction need it even on the reduced-precision path).
#include <math.h>

#include "wpcd_internal.cuh"
#include "logtab.h"

namespace wpcd {

constexpr int kTThreads = 256;

// ---------------------------------------------------------------------------------------------
// Energy plan: per channel and energy, the free bin holding p(E) and the
// segment of interpolation points used for interpolation; per channel, the distinct bins
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
            hi = N - 1;  // largest j whose interpolation point is <= p (or -1)
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (ip_point(ch.kb, mid, plan.ip_frac) <= p) lo = mid;
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
    k_plan<<<dim3(n_ch, n_plans), 256, 0, counted(st)>>>(chans_dev, n_ch, maxN, e_lab, n_E, plan, err);
    return cudaGetLastError();
}

// Natural logarithm of a positive double, table-driven after P. T. P. Tang,
// "Table-driven implementation of the logarithm function in IEEE
// floating-point arithmetic", ACM TOMS 16 (1990): x = 2^k m with m in [1, 2),
// F = 1 + j/256 the nearest table point (j = 256 is folded into k + 1 and
// F = 1), u = (m - F) / F with |u| <= 2^-9, and
//     log x = k log 2 + log F + log1p(u),
// log 2 and log F as double-double table values (logtab.h) and log1p(u) from
// its series through u^6 (truncation |u|^7 / 7 < 2^-65).  Below 1 ulp in a
// CPU emulation with exact FMA; 13 FP64 operations.  The resolvent evaluates
// (m + 1)(n + 1) of these per solve on GB300's narrow FP64 pipe; against the
// library log this took the T phase of a 4096-sample step from 28.9 to 21.9 ms.
// Zero, subnormal, infinite and NaN arguments take the library log.
__device__ __forceinline__ double wlog(double x)
{
    const long long b = __double_as_longlong(x);
    const int be = (int)(b >> 52);  // biased exponent; negative for a negative x
    if (be <= 0 || be >= 0x7FF) return log(x);
    const long long mant = b & 0x000FFFFFFFFFFFFFll;
    int j = (int)((mant + (1ll << 43)) >> 44);  // nearest of 256 (m - 1), 0 .. 256
    int k = be - 1023;
    long long mb = mant | 0x3FF0000000000000ll;  // m
    if (j == 256) {  // m / 2 in [1 - 2^-10, 1) against F = 1
        mb -= 1ll << 52;
        ++k;
        j = 0;
    }
    const LogEntry t = kLogTab[j];
    const double f = __longlong_as_double(mb) - __longlong_as_double(0x3FF0000000000000ll + ((long long)j << 44));
    const double u = f * t.inv;  // f is exact: m and F are within a factor of two
    const double kd = (double)k;
    const double c = fma(u, fma(u, fma(u, fma(u, -1.0 / 6.0, 0.2), -0.25), 1.0 / 3.0), -0.5);
    const double lo = fma(kd, kLn2Lo, t.lo);
    return fma(kd, kLn2Hi, t.hi) + (u + fma(u * u, c, lo));
}

__device__ __forceinline__ double xlogabs(double d) { return d == 0.0 ? 0.0 : d * wlog(fabs(d)); }

// ---------------------------------------------------------------------------------------------
// On-shell T.  One CTA per (sample, channel).
//  - SWP boundaries (Eq. "pseudostate wave packet boundaries"): the positive
//    eigenvalues of each branch give B_1 = 0, B_i = (e_{i-1}+e_i)/2,
//    B_{m+1} = e_m + (B_m - B_{m-1})/2.  Coupled channels: the positive
//    eigenvalues, sorted, are dealt to the two branches alternately from the
//    top (largest -> branch 1).
//  - for each item (a needed free bin i, or a requested energy E in free bin i):
//    the VC rows R_as = sum_j V_(a,i),j C_js and the resolvent
//      MODE 0 (free-bin average, App. B with the sign of W corrected): over
//        [Ea, Eb] = [E_i, E_{i+1}],
//        gbar_s = [X(Eb,B_s) - X(Ea,B_s) - X(Eb,B_s+1) + X(Ea,B_s+1)]/(dE dB)
//                 - i pi |[Ea,Eb] ^ [B_s,B_s+1]| / (dE dB),  X(a,b) = (a-b) ln|a-b|,
//        or ln((Eb - e_b)/(Ea - e_b))/dE for a bound state e_b < 0;
//      MODE 1 (SWP-bin average, App. B as printed): the same over SWP bin i,
//        [Ea, Eb] = [B_i, B_{i+1}] (uncoupled channels without bound states);
//      MODE 2 (point resolvent, App. B): at E itself,
//        g_s = [ln|(E - B_s)/(E - B_s+1)| - i pi 1{E in [B_s, B_s+1]}] / dB,
//        or 1/(E - e_b);
//    then T_ab = V_(a,i),(b,i) + sum_s R_as g_s R_bs.
//  - continuum T: T f(q)^2 / (N_i q^2) at q = the bin's interpolation point (modes 0, 1;
//    the midpoint unless the caller set another, Sec. 5.1.1)
//    or q = p(E) (mode 2); S = 1 - 2 pi i mu q T; phases (Stapp for coupled
//    channels).
// Averaged modes visit the needed bins in ascending order, so the X(E_{i+1}, B)
// of one bin are the X(E_i, B) of the next whenever the bins are adjacent.
// VCID: the VC rows from the eigen-equation.  H0 is diagonal in the free
// packet basis, so V C = H C - H0 C = C diag(e) - H0 C, i.e.
//     R_as = C_(a,i),s (e_s - h0_i),
// exact for exact eigenpairs; its error is the eigen residual (~u ||H||
// absolute).  Used on the mixed path, whose eigenpairs are refined to FP64
// residuals; the FP64 path keeps the explicit products (their error scales with
// ||V|| rather than ||H||, which holds the relative accuracy of small T).
// Output, 8 doubles (complex 2 x 2) and 3 phases per item: modes 0, 1 at
// [S][n_ch][stride = maxN][bin], mode 2 at [S][n_ch][stride = n_E][energy].
// ---------------------------------------------------------------------------------------------
template <bool VCID, int MODE>
__global__ void __launch_bounds__(kTThreads, 5) k_tmat(const ChanDev *chans, int n_ch, int n_terms, const double *coeffs,
                                                    const double *eps_all, const double *C_all, PlanDev plan,
                                                    int n_E, int stride, double *tout, double *phout, int *err)
{
    const int c = blockIdx.x % n_ch, smp = blockIdx.x / n_ch;
    const ChanDev ch = chans[c];
    const int n = ch.n, N = ch.N, K = ch.K;
    const int tid = threadIdx.x, nt = blockDim.x;
    if ((size_t)dyn_smem_bytes() < tbin_smem_doubles(n) * sizeof(double) || nt != kTThreads) {  // launch/layout mismatch
        if (tid == 0) record_error(err, kDevBadSize);
        return;
    }
    extern __shared__ double sm[];
    double *eps = sm;               // n
    double *Eb = eps + n;           // 2 x n   branch members
    double *Bb = Eb + 2 * n;        // 2 x (n+1) branch boundaries
    double *lo = Bb + 2 * (n + 1);  // n  lower SWP boundary of eigenvalue s
    double *hi = lo + n;            // n  upper
    double *idB = hi + n;           // n  1 / (hi - lo)
    double *XA = idB + n;           // n+4  D(B) = X(E_{i+1}, B) - X(E_i, B) per boundary slot (averaged modes)
    double *XB = XA + n + 4;        // n+4  X(E_{i+1}, B)
    double *vrow = XB + n + 4;      // K x n
    double *R = vrow + 2 * n;       // K x n
    double *red = R + 2 * n;        // 8   the six T sums
    double *rs = red + 8;           // 6 x kTThreads  per-thread terms of the six sums
    double *vd = rs + 6 * kTThreads;  // K x K diagonal V entries
    // averaged modes, per needed bin (the plan's list order): its edges, 1/dE and the
    // continuum factor f^2 / (N_i q^2), formed once per item instead of per thread and bin
    double *binA = vd + 4, *binB = binA + N, *binI = binB + N, *binF = binI + N;
    int *bini = reinterpret_cast<int *>(binF + N);
    __shared__ int s_nb, s_bad;

    const double *eg = eps_all + ch.eps_off + (size_t)smp * n;
    const double *C = C_all + ch.c_off + (size_t)smp * n * n;
    const double *cf = coeffs ? coeffs + (size_t)smp * (n_terms - 1) : nullptr;
    const int ps = plan_of(plan, smp);
    const size_t pc = (size_t)ps * n_ch + c;
    const int cnt = MODE == 2 ? plan_nE(plan, ps, n_E) : plan.cnt[pc];
    const size_t obase = ((size_t)smp * n_ch + c) * stride;

    if (tid == 0) { s_nb = 0; s_bad = 0; }
    for (int s = tid; s < n; s += nt) eps[s] = eg[s];
    __syncthreads();
    for (int s = tid; s < n; s += nt)
        if (eps[s] < 0.0 && (s == n - 1 || !(eps[s + 1] < 0.0))) s_nb = s + 1;
    __syncthreads();
    const int nb = s_nb, P = n - nb;
    if (MODE == 1 && (K != 1 || nb != 0)) {  // SWP-bin averaging is defined for these only
        for (int ii = tid; ii < cnt; ii += nt) {
            const int i = plan.list[pc * stride + ii];
            for (int k = 0; k < 8; ++k) tout[(obase + i) * 8 + k] = __longlong_as_double(0x7ff8000000000000ll);
            for (int k = 0; k < 3; ++k) phout[(obase + i) * 3 + k] = __longlong_as_double(0x7ff8000000000000ll);
        }
        if (tid == 0) record_error(err, kDevMode);
        return;
    }
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
        idB[s] = 1.0 / (hi[s] - lo[s]);
    }
    __syncthreads();

    if (MODE != 2) {
        for (int ii = tid; ii < cnt; ii += nt) {
            const int i = plan.list[pc * stride + ii];
            double a, b;
            if (MODE == 1) {
                a = Bb[i];
                b = Bb[i + 1];
            } else {
                a = ch.kb[i] * ch.kb[i] / (2.0 * kMu);
                b = ch.kb[i + 1] * ch.kb[i + 1] / (2.0 * kMu);
            }
            const double q = ip_point(ch.kb, i, plan.ip_frac);
            const double Ni = ch.wp_kind == 0 ? (ch.kb[i + 1] - ch.kb[i])
                                              : (ch.kb[i + 1] * ch.kb[i + 1] - ch.kb[i] * ch.kb[i]) / (2.0 * kMu);
            const double f2 = ch.wp_kind == 0 ? 1.0 : q / kMu;
            bini[ii] = i;
            binA[ii] = a;
            binB[ii] = b;
            binI[ii] = 1.0 / (b - a);
            binF[ii] = f2 / (Ni * q * q);
        }
        __syncthreads();
    }

    const int dstride = (K == 2) ? (n >> 1) + 2 : n + 1;  // boundary slots per branch (K * dstride <= n + 4)
    int prev = -2;                                          // bin whose upper-edge X values sit in XB
    for (int ii = 0; ii < cnt; ++ii) {
        int i;
        double Ea = 0.0, Ebn = 0.0, E = 0.0, p = 0.0;
        if (MODE == 2) {
            i = plan.bin[pc * n_E + ii];
            p = plan.pE[(size_t)ps * n_E + ii];
            E = p * p / (2.0 * kMu);
        } else {
            i = bini[ii];
            Ea = binA[ii];
            Ebn = binB[ii];
        }
        // this bin's eigenvector rows, first element per thread issued early so
        // that the load overlaps the logarithms below
        const double *C0 = C + (size_t)i * n, *C1 = C + (size_t)(N + i) * n;
        double c0pre = 0.0, c1pre = 0.0;
        if (VCID && tid < n) {
            c0pre = C0[tid];
            if (K == 2) c1pre = C1[tid];
        }
        // the diagonal entries V_(a,i),(b,i) of V = V0 + sum_t c_t V_t: warp w < K^2
        // forms entry w, lane l its terms l, l + 32, ... (loads in flight during the
        // logarithms below, summed with a butterfly after them)
        double vterm = 0.0;
        if (VCID && (tid >> 5) < K * K) {
            const int w = tid >> 5, a = w / K, bb = w - a * K;
            const size_t off = (size_t)(a * N + i) * n + bb * N + i;
            for (int t = tid & 31; t < n_terms; t += 32) {
                const double v = ch.V[(size_t)t * n * n + off];
                vterm += t == 0 ? v : cf[t - 1] * v;
            }
        }
        if (MODE != 2) {
            const bool reuse = (i == prev + 1);
            if (reuse) {  // the previous upper edge is this lower edge
                double *t = XA;
                XA = XB;
                XB = t;
            }
            // XB = X(E_{i+1}, B); XA becomes D(B) = X(E_{i+1}, B) - X(E_i, B) (its
            // X(E_i, B) is either the previous bin's XB or computed here)
            for (int e = tid; e < K * dstride; e += nt) {
                const int b = e / dstride, pos = e - b * dstride;
                if (pos <= mcount[b]) {
                    const double B = Bb[b * (n + 1) + pos];
                    const double xb = xlogabs(Ebn - B);
                    XB[e] = xb;
                    XA[e] = xb - (reuse ? XA[e] : xlogabs(Ea - B));
                }
            }
        }
        if (VCID) {
            if ((tid >> 5) < K * K) {  // warp-uniform
                for (int o = 16; o > 0; o >>= 1) vterm += __shfl_xor_sync(0xffffffffu, vterm, o);
                if ((tid & 31) == 0) vd[tid >> 5] = vterm;
            }
        } else {
            // rows (a, i) of V, then R = V_rows C
            for (int e = tid; e < K * n; e += nt) {
                const int a = e / n, jj = e - a * n;
                const size_t off = (size_t)(a * N + i) * n + jj;
                double v = ch.V[off];
                for (int t = 1; t < n_terms; ++t) v = fma(cf[t - 1], ch.V[(size_t)t * n * n + off], v);
                vrow[a * n + jj] = v;
            }
            __syncthreads();
            for (int e = tid; e < K * n; e += nt) {
                const int a = e / n, s = e - a * n;
                const double *vr = vrow + a * n;
                double acc = 0.0;
                for (int j = 0; j < n; ++j) acc = fma(vr[j], C[(size_t)j * n + s], acc);
                R[a * n + s] = acc;
            }
        }
        __syncthreads();
        // thread 0 keeps the diagonal V entries in registers: the next item rewrites them
        double v00 = 0.0, v01 = 0.0, v10 = 0.0, v11 = 0.0;
        if (tid == 0) {
            if (VCID) {
                v00 = vd[0];
                if (K == 2) { v01 = vd[1]; v10 = vd[2]; v11 = vd[3]; }
            } else {
                v00 = vrow[i];
                if (K == 2) { v01 = vrow[N + i]; v10 = vrow[n + i]; v11 = vrow[n + N + i]; }
            }
        }
        const double idE = MODE == 2 ? 0.0 : binI[ii];
        const double h0i = VCID ? ch.h0[i] : 0.0;
        double acc[6] = {0, 0, 0, 0, 0, 0};  // (00 re, im), (01 re, im), (11 re, im)
        for (int s = tid; s < n; s += nt) {
            double gre, gim = 0.0;
            if (s < nb) {
                gre = MODE == 2 ? 1.0 / (E - eps[s]) : wlog((Ebn - eps[s]) / (Ea - eps[s])) * idE;
            } else {
                const int d = s - nb;
                const int b = (K == 2) ? (((n - 1 - s) & 1) == 0 ? 1 : 0) : 0;
                const int q = b * dstride + ((K == 2) ? d / 2 : d);
                if (MODE == 2) {  // the log of the ratio: no cancellation far from the bin
                    gre = wlog(fabs((E - lo[s]) / (E - hi[s]))) * idB[s];
                    if (E >= lo[s] && E <= hi[s]) gim = -kPi * idB[s];
                } else {
                    const double w = idB[s] * idE;  // 1 / (dE dB)
                    gre = (XA[q] - XA[q + 1]) * w;  // D(B_s) - D(B_s+1)
                    const double l = Ea > lo[s] ? Ea : lo[s], h = Ebn < hi[s] ? Ebn : hi[s];
                    if (h > l) gim = -kPi * (h - l) * w;
                }
            }
            double r0, r1 = 0.0;
            if (VCID) {
                const double de = eps[s] - h0i;
                r0 = (s == tid ? c0pre : C0[s]) * de;
                if (K == 2) r1 = (s == tid ? c1pre : C1[s]) * de;
            } else {
                r0 = R[s];
                if (K == 2) r1 = R[n + s];
            }
            const double r00 = r0 * r0;
            acc[0] = fma(r00, gre, acc[0]);
            if (K == 2) {
                acc[2] = fma(r0 * r1, gre, acc[2]);
                acc[4] = fma(r1 * r1, gre, acc[4]);
            }
            if (gim != 0.0) {  // only the few states whose SWP bin overlaps the energy (range)
                acc[1] = fma(r00, gim, acc[1]);
                if (K == 2) {
                    acc[3] = fma(r0 * r1, gim, acc[3]);
                    acc[5] = fma(r1 * r1, gim, acc[5]);
                }
            }
        }
        // the six sums over the CTA: every thread's terms go to shared memory and
        // warp k adds up sum k (nt/32 loads and a 5-step butterfly per thread), so
        // the FP64 adds are ~nt per sum instead of a 6-value butterfly in every warp
        const int nv = K == 2 ? 6 : 2;
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (k < nv) rs[k * kTThreads + tid] = acc[k];
        __syncthreads();
        if ((tid >> 5) < nv) {
            const int k = tid >> 5, ln = tid & 31;
            double t = 0.0;
            for (int j = ln; j < nt; j += 32) t += rs[k * kTThreads + j];
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (ln == 0) red[k] = t;
        }
        __syncthreads();
        prev = i;
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < 6; ++k) acc[k] = (k < nv) ? red[k] : 0.0;
            double fac;
            if (MODE == 2) {
                const double Ni = ch.wp_kind == 0 ? (ch.kb[i + 1] - ch.kb[i])
                                                  : (ch.kb[i + 1] * ch.kb[i + 1] - ch.kb[i] * ch.kb[i]) / (2.0 * kMu);
                const double f2 = ch.wp_kind == 0 ? 1.0 : p / kMu;
                fac = f2 / (Ni * p * p);
            } else {
                fac = binF[ii];
            }
            double T[8];  // complex 2x2, row-major
            T[0] = fac * (v00 + acc[0]);
            T[1] = fac * acc[1];
            if (K == 2) {
                T[2] = fac * (v01 + acc[2]);
                T[3] = fac * acc[3];
                T[4] = fac * (v10 + acc[2]);
                T[5] = fac * acc[3];
                T[6] = fac * (v11 + acc[4]);
                T[7] = fac * acc[5];
            } else {
                T[2] = T[3] = T[4] = T[5] = T[6] = T[7] = 0.0;
            }
            double *to = tout + (obase + (MODE == 2 ? ii : i)) * 8;
            for (int k = 0; k < 8; ++k) to[k] = T[k];
        }
        // no trailing barrier: the next item writes X, V, R and the warp sums only
        // after its first barrier, which thread 0 reaches after reading them
    }
    // S and the phases of every item, one item per thread (their T were
    // written above by thread 0 of this CTA)
    __syncthreads();
    for (int ii = tid; ii < cnt; ii += nt) {
        const int slot = MODE == 2 ? ii : plan.list[pc * stride + ii];
        const int i = MODE == 2 ? plan.bin[pc * n_E + ii] : slot;
        const double q = MODE == 2 ? plan.pE[(size_t)ps * n_E + ii] : ip_point(ch.kb, i, plan.ip_frac);
        phases_of_T(K, q, tout + (obase + slot) * 8, phout + (obase + slot) * 3);
    }
}

size_t tbin_smem_bytes(int nmax) { return tbin_smem_doubles(nmax) * sizeof(double); }

template <bool VCID, int MODE>
static void launch_tmat_t(const ChanDev *chans_dev, int n_ch, int n_samples, int n_terms, const double *coeffs,
                          const double *eps_all, const double *C_all, PlanDev plan, int n_E, int stride,
                          size_t smem, double *tout, double *phout, int *err, cudaStream_t st)
{
    raise_smem_limit((const void *)k_tmat<VCID, MODE>, smem);
    k_tmat<VCID, MODE><<<(unsigned)(n_samples * n_ch), kTThreads, smem, counted(st)>>>(chans_dev, n_ch, n_terms, coeffs, eps_all,
                                                                              C_all, plan, n_E, stride, tout, phout,
                                                                              err);
}

cudaError_t launch_tbin(const ChanDev *chans_dev, int n_ch, int n_samples, int n_terms, const double *coeffs,
                        const double *eps_all, const double *C_all, PlanDev plan, int maxN, int n_E, double *tout,
                        double *phout, int *err, cudaStream_t st, bool vc_identity, int mode)
{
    if (mode < 0 || mode > 2) return cudaErrorInvalidValue;
    const size_t smem = tbin_smem_bytes(2 * maxN);
    const int stride = mode == 2 ? n_E : maxN;
#define WPCD_TMAT(V, M) \
    launch_tmat_t<V, M>(chans_dev, n_ch, n_samples, n_terms, coeffs, eps_all, C_all, plan, n_E, stride, smem, tout, phout, err, st)
    if (vc_identity) {
        if (mode == 0) WPCD_TMAT(true, 0);
        else if (mode == 1) WPCD_TMAT(true, 1);
        else WPCD_TMAT(true, 2);
    } else {
        if (mode == 0) WPCD_TMAT(false, 0);
        else if (mode == 1) WPCD_TMAT(false, 1);
        else WPCD_TMAT(false, 2);
    }
#undef WPCD_TMAT
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// T at the requested energies: the value of the bin holding p(E) (averaged
// resolvents, stride = maxN), or the energy's own value (point resolvent,
// direct, stride = n_E).  t_out: [S][n_ch][n_E][2][2] complex.
// ---------------------------------------------------------------------------------------------
__global__ void k_gather_t(int n_ch, int n_samples, int n_E, int stride, bool direct, PlanDev plan,
                           const double *tbin, double *t_out)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)n_samples * n_ch * n_E;
    if (idx >= total) return;
    const int e = (int)(idx % n_E);
    const size_t sc = idx / n_E;
    const int c = (int)(sc % n_ch);
    const int ps = plan_of(plan, (int)(sc / n_ch));
    if (e >= plan_nE(plan, ps, n_E)) return;
    const int slot = direct ? e : plan.bin[((size_t)ps * n_ch + c) * n_E + e];
    const double *src = tbin + (sc * stride + slot) * 8;
    double *dst = t_out + idx * 8;
    const double2 *s2 = reinterpret_cast<const double2 *>(src);
    double2 *d2 = reinterpret_cast<double2 *>(dst);
#pragma unroll
    for (int k = 0; k < 4; ++k) d2[k] = s2[k];
}

// The T kernel's logarithm applied elementwise, for tests against other implementations.
__global__ void k_wlog(const double *x, double *y, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = wlog(x[i]);
}

cudaError_t launch_wlog(const double *x, double *y, int n, cudaStream_t st)
{
    if (n > 0) k_wlog<<<(n + 255) / 256, 256, 0, counted(st)>>>(x, y, n);
    return cudaGetLastError();
}

cudaError_t launch_gather_t(const ChanDev *chans_dev, int n_ch, int n_samples, int n_E, int maxN, PlanDev plan,
                            const double *tbin, double *t_out, cudaStream_t st, bool direct)
{
    (void)chans_dev;
    const size_t total = (size_t)n_samples * n_ch * n_E;
    k_gather_t<<<(unsigned)((total + 255) / 256), 256, 0, counted(st)>>>(n_ch, n_samples, n_E, direct ? n_E : maxN, direct,
                                                                plan, tbin, t_out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Phases interpolated linearly in p between the interpolation points (the
// midpoints unless the caller set another) of the segment j, j+1 (extended
// past the end points), after moving delta_{j+1} by a
// multiple of 180 deg to within 90 deg of delta_j; result mapped to
// (-90, 90]; with the point resolvent (direct) the phases at p(E) itself.
// Total cross section sigma = pi/(2p^2) sum (2J+1) sum_l Re(1 - S_ll) over the
// np channels (tz = 0), with S rebuilt from those Stapp parameters.  One
// thread per (sample, energy).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double wrap90(double d)
{
    if (!isfinite(d)) return d;
    while (d > 90.0) d -= 180.0;
    while (d <= -90.0) d += 180.0;
    return d;
}

__global__ void k_observables(const ChanDev *chans, int n_ch, int n_samples, int n_E, int stride, bool direct,
                              PlanDev plan, const double *phbin, double *delta, double *sigma)
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
        const double *ph = phbin + (((size_t)smp * n_ch + c) * stride) * 3;
        double out[3];
        if (direct) {
            for (int k = 0; k < 3; ++k) out[k] = ph[3 * e + k];
        } else {
            const int j = plan.brk[((size_t)ps * n_ch + c) * n_E + e];
            const double q0 = ip_point(ch.kb, j, plan.ip_frac), q1 = ip_point(ch.kb, j + 1, plan.ip_frac);
            const double w = (p - q0) / (q1 - q0);
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
                               const double *phbin, double *delta, double *sigma, cudaStream_t st, bool direct)
{
    const size_t total = (size_t)n_samples * n_E;
    k_observables<<<(unsigned)((total + 127) / 128), 128, 0, counted(st)>>>(chans_dev, n_ch, n_samples, n_E,
                                                                    direct ? n_E : maxN, direct, plan, phbin, delta,
                                                                    sigma);
    return cudaGetLastError();
}

}  // namespace wpcd
