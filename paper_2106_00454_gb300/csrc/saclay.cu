// saclay.cu -- spin observables of np scattering (App. A) from the phase
// shifts: the M-matrix partial-wave expansion, the Saclay amplitudes a..e and
// dsigma/dOmega, batched over (sample, energy, angle).
//
// With the incoming momentum along z and phi = 0, momentum-space partial waves
// and every np channel once,
//   M^s_{m'm}(theta) = sqrt(4 pi)/(2 i p) sum_{J,l,l'} sqrt(2l+1)
//       C(l' (m-m') s m' | J m) C(l 0 s m | J m) (S_{l'l} - delta_{l'l}) Y_{l'}^{m-m'}(theta, 0),
// S rebuilt from the (Stapp) phases.  The coupling products of the sum are
// tabulated per channel on the host (Clebsch-Gordan by Racah's formula); the
// spherical harmonics follow from the associated-Legendre recurrences.  M is
// taken to the product spin basis and the amplitudes are its coefficients in
//   M = [(a+b) + (a-b)(s1.n)(s2.n) + (c+d)(s1.m)(s2.m) + (c-d)(s1.l)(s2.l) + e(s1+s2).n] / 2,
// l, m, n along p + p', p - p', p x p'; dsigma/dOmega = Tr(M M^+)/4.
#include <math.h>

#include "wpcd_internal.cuh"

namespace wpcd {

struct Cplx {
    double re, im;
};
__device__ __forceinline__ Cplx cmul(Cplx a, Cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ Cplx cadd(Cplx a, Cplx b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ Cplx cscale(Cplx a, double s) { return {a.re * s, a.im * s}; }

// Y_l^m(theta, 0), Condon-Shortley phase, |m| <= 2, l <= kSacLmax.
__device__ double ylm0(int l, int m, double x, double s)
{
    const int am = m < 0 ? -m : m;
    if (am > l) return 0.0;
    double pmm = 1.0;
    for (int i = 1; i <= am; ++i) pmm *= (2.0 * i - 1.0) * s;
    double plm = pmm;
    if (l > am) {
        double p0 = pmm, p1 = x * (2.0 * am + 1.0) * pmm;
        plm = p1;
        for (int ll = am + 2; ll <= l; ++ll) {
            const double pn = ((2.0 * ll - 1.0) * x * p1 - (ll + am - 1.0) * p0) / (ll - am);
            p0 = p1;
            p1 = pn;
            plm = pn;
        }
    }
    // sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!)
    double ratio = 1.0;
    for (int k = l - am + 1; k <= l + am; ++k) ratio /= k;
    double y = sqrt((2.0 * l + 1.0) / (4.0 * kPi) * ratio) * plm;
    if (am & 1) y = -y;            // (-1)^m for m >= 0
    if (m < 0 && (am & 1)) y = -y;  // Y_l^{-m} = (-1)^m Y_l^m at phi = 0
    return y;
}

// One thread per (sample, energy, angle).  tab: per channel [2][2][3][3]
// coupling products (l' block, l block, m' + 1, m + 1), zero where not allowed;
// lblk: per channel the two l values; delta [S][n_ch][n_E][3] degrees.
__global__ void k_saclay(const SacChanDev *chans, int n_ch, int n_samples, int n_E, const double *e_lab,
                         const double *delta, int n_th, const double *theta, double *abcde, double *dsig)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n_samples * n_E * n_th) return;
    const int t = (int)(idx % n_th);
    const size_t se = idx / n_th;
    const int e = (int)(se % n_E), smp = (int)(se / n_E);
    const double p = sqrt(kMn * e_lab[e] / 2.0) / kHbarc;
    const double th = theta[t], x = cos(th), sn = sin(th);
    const double rad = kPi / 180.0;
    Cplx M0 = {0.0, 0.0}, M1[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) M1[a][b] = {0.0, 0.0};
    for (int c = 0; c < n_ch; ++c) {
        const SacChanDev ch = chans[c];
        if (ch.tz != 0) continue;
        const double *ph = delta + (((size_t)smp * n_ch + c) * n_E + e) * 3;
        Cplx S[2][2];
        if (ch.K == 1) {
            S[0][0] = {cos(2.0 * ph[0] * rad), sin(2.0 * ph[0] * rad)};
        } else {
            const double dm = ph[0] * rad, dp = ph[1] * rad, e2 = 2.0 * ph[2] * rad, ce = cos(e2), se2 = sin(e2);
            S[0][0] = {ce * cos(2.0 * dm), ce * sin(2.0 * dm)};
            S[1][1] = {ce * cos(2.0 * dp), ce * sin(2.0 * dp)};
            // i sin(2 eps) e^{i (dm + dp)}
            S[0][1] = S[1][0] = {-se2 * sin(dm + dp), se2 * cos(dm + dp)};
        }
        for (int ip = 0; ip < ch.K; ++ip)
            for (int il = 0; il < ch.K; ++il) {
                Cplx amp = S[ip][il];
                if (ip == il) amp.re -= 1.0;
                const int lp = ch.l[ip];
                for (int mp = -ch.s; mp <= ch.s; ++mp)
                    for (int m = -ch.s; m <= ch.s; ++m) {
                        const double w = ch.tab[((ip * 2 + il) * 3 + (mp + 1)) * 3 + (m + 1)];
                        if (w == 0.0) continue;
                        const Cplx v = cscale(amp, w * ylm0(lp, m - mp, x, sn));
                        if (ch.s == 0) M0 = cadd(M0, v);
                        else M1[mp + 1][m + 1] = cadd(M1[mp + 1][m + 1], v);
                    }
            }
    }
    // / (2 i p)
    const double f = 1.0 / (2.0 * p);
    auto div2ip = [f](Cplx z) { return Cplx{z.im * f, -z.re * f}; };
    M0 = div2ip(M0);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) M1[a][b] = div2ip(M1[a][b]);
    // product basis uu, ud, du, dd: |1,1> = uu, |1,0> = (ud+du)/sqrt2, |1,-1> = dd, |0,0> = (ud-du)/sqrt2
    const double h = 0.70710678118654752440;
    const double U[4][4] = {{1, 0, 0, 0}, {0, h, 0, h}, {0, h, 0, -h}, {0, 0, 1, 0}};  // columns: (1,1),(1,0),(1,-1),(0,0)
    Cplx Mc[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) Mc[i][j] = {0.0, 0.0};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Mc[2 - a][2 - b] = M1[a][b];
    Mc[3][3] = M0;
    Cplx M[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            Cplx acc = {0.0, 0.0};
            for (int k = 0; k < 4; ++k) {
                if (U[i][k] == 0.0) continue;
                for (int l = 0; l < 4; ++l)
                    if (U[j][l] != 0.0) acc = cadd(acc, cscale(Mc[k][l], U[i][k] * U[j][l]));
            }
            M[i][j] = acc;
        }
    // spin operators: s.v = [[vz, vx - i vy], [vx + i vy, -vz]]
    const double ch2 = cos(0.5 * th), sh2 = sin(0.5 * th);
    const double lv[3] = {sh2, 0.0, ch2}, mv[3] = {-ch2, 0.0, sh2}, nv[3] = {0.0, 1.0, 0.0};
    auto pauli = [](const double *v, Cplx P[2][2]) {
        P[0][0] = {v[2], 0.0};
        P[0][1] = {v[0], -v[1]};
        P[1][0] = {v[0], v[1]};
        P[1][1] = {-v[2], 0.0};
    };
    Cplx Pl[2][2], Pm[2][2], Pn[2][2];
    pauli(lv, Pl);
    pauli(mv, Pm);
    pauli(nv, Pn);
    // Tr(M (A (x) B)) = sum_{i,j,k,l} M[2j+l][2i+k] A[i][j] B[k][l]
    auto tr_kron = [&](Cplx A[2][2], Cplx B[2][2]) {
        Cplx acc = {0.0, 0.0};
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
                for (int k = 0; k < 2; ++k)
                    for (int l = 0; l < 2; ++l) acc = cadd(acc, cmul(M[2 * j + l][2 * i + k], cmul(A[i][j], B[k][l])));
        return acc;
    };
    Cplx Id[2][2] = {{{1.0, 0.0}, {0.0, 0.0}}, {{0.0, 0.0}, {1.0, 0.0}}};
    const Cplx apb = cscale(tr_kron(Id, Id), 0.5), amb = cscale(tr_kron(Pn, Pn), 0.5),
               cpd = cscale(tr_kron(Pm, Pm), 0.5), cmd = cscale(tr_kron(Pl, Pl), 0.5),
               ee = cscale(cadd(tr_kron(Pn, Id), tr_kron(Id, Pn)), 0.25);
    const Cplx out[5] = {cscale(cadd(apb, amb), 0.5), cscale(cadd(apb, cscale(amb, -1.0)), 0.5),
                         cscale(cadd(cpd, cmd), 0.5), cscale(cadd(cpd, cscale(cmd, -1.0)), 0.5), ee};
    if (abcde)
        for (int k = 0; k < 5; ++k) {
            abcde[idx * 10 + 2 * k] = out[k].re;
            abcde[idx * 10 + 2 * k + 1] = out[k].im;
        }
    if (dsig) {
        double tr = 0.0;
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) tr += M[i][j].re * M[i][j].re + M[i][j].im * M[i][j].im;
        dsig[idx] = 0.25 * tr * 10.0;  // fm^2 -> mb
    }
}

cudaError_t launch_saclay(const SacChanDev *chans_dev, int n_ch, int n_samples, int n_E, const double *e_lab,
                          const double *delta, int n_th, const double *theta, double *abcde, double *dsig,
                          cudaStream_t st)
{
    const size_t total = (size_t)n_samples * n_E * n_th;
    k_saclay<<<(unsigned)((total + 127) / 128), 128, 0, counted(st)>>>(chans_dev, n_ch, n_samples, n_E, e_lab, delta, n_th,
                                                               theta, abcde, dsig);
    return cudaGetLastError();
}

}  // namespace wpcd
