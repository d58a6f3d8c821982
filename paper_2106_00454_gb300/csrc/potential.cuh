// potential.cuh -- the built-in potentials' partial-wave terms at one momentum
// pair (p', p), shared by the wave-packet projection and the MI grid.
//
// Yamaguchi (rank 1, S wave): V = lambda / ((p'^2 + beta^2)(p^2 + beta^2)).
// Synthetic Yukawa + contact set (14 unit terms and V0 = sum_a gp[4 + a] u_a):
// Yukawa radial forms 1/(q^2 + m^2) projected on the partial waves by the
// 96-point angle rule, I_L[m](p', p) = 2 pi sum_x w_x P_L(x) / (p^2 + p'^2 -
// 2 p p' x + m^2), with the LSJ factors of the central, spin-spin, spin-orbit
// and tensor operators, nine partial-wave contacts, all times the Gaussian
// regulator exp(-(p'^2 + p^2) / Lambda^2).
#pragma once

#include "wpcd_internal.cuh"

namespace wpcd {

constexpr int kLmaxReg = 10;  // angle integrals kept in registers: L = 0..10 (J <= 8)

__device__ __forceinline__ double ls_factor(int s, int J, int l)
{
    return 0.5 * (J * (J + 1.0) - l * (l + 1.0) - s * (s + 1.0));
}

__device__ __forceinline__ double s12_factor(int s, int J, int lp, int l)
{
    if (s != 1) return 0.0;
    if (lp == l) {
        if (l == J) return 2.0;
        if (l == J - 1) return -2.0 * (J - 1.0) / (2.0 * J + 1.0);
        if (l == J + 1) return -2.0 * (J + 2.0) / (2.0 * J + 1.0);
        return 0.0;
    }
    if ((lp == J - 1 && l == J + 1) || (lp == J + 1 && l == J - 1)) return 6.0 * sqrt(J * (J + 1.0)) / (2.0 * J + 1.0);
    return 0.0;
}

// w_x P_L(x) for L = 0..Lm and the nodes x, into shared tables (all threads of
// the CTA take part; the caller synchronises afterwards).
__device__ __forceinline__ void angle_tables(const double *angx, const double *angw, int Lm,
                                             double (*wpl)[kLmaxReg + 1], double *ax)
{
    for (int x = threadIdx.x; x < kAngleQ; x += blockDim.x) {
        double xv = angx[x], p0 = 1.0, p1 = xv;
        ax[x] = xv;
        wpl[x][0] = angw[x];
        if (Lm >= 1) wpl[x][1] = angw[x] * xv;
        for (int L = 2; L <= Lm; ++L) {
            double p2 = ((2.0 * L - 1.0) * xv * p1 - (L - 1.0) * p0) / L;
            p0 = p1;
            p1 = p2;
            wpl[x][L] = angw[x] * p2;
        }
    }
}

// The three Yukawa angle integrals I_L[m_1..3](p', p), L = 0..Lm (zero above),
// and the regulator R.
__device__ __forceinline__ void yukawa_angle_integrals(const double *gp, const double (*wpl)[kLmaxReg + 1],
                                                       const double *ax, int Lm, double pp, double p, double *I1,
                                                       double *I2, double *I3, double &R)
{
    const double m1 = gp[0], m2 = gp[1], m3 = gp[2], Lam = gp[3];
#pragma unroll
    for (int L = 0; L <= kLmaxReg; ++L) I1[L] = I2[L] = I3[L] = 0.0;
    const double A0 = pp * pp + p * p, B = 2.0 * pp * p;
    for (int x = 0; x < kAngleQ; ++x) {
        double d = A0 - B * ax[x];
        double F1 = 1.0 / (d + m1 * m1), F2 = 1.0 / (d + m2 * m2), F3 = 1.0 / (d + m3 * m3);
#pragma unroll
        for (int L = 0; L <= kLmaxReg; ++L) {
            if (L <= Lm) {
                double wv = wpl[x][L];
                I1[L] = fma(wv, F1, I1[L]);
                I2[L] = fma(wv, F2, I2[L]);
                I3[L] = fma(wv, F3, I3[L]);
            }
        }
    }
#pragma unroll
    for (int L = 0; L <= kLmaxReg; ++L) {
        I1[L] *= 2.0 * kPi;
        I2[L] *= 2.0 * kPi;
        I3[L] *= 2.0 * kPi;
    }
    R = exp(-(pp * pp + p * p) / (Lam * Lam));
}

// Synthetic Yukawa + contact set: tv[0] = V0, tv[1..14] = the unit terms u_a
// (tv must hold kMaxTerms zeros on entry).
__device__ __forceinline__ void yukawa_terms(const double *gp, int s, int J, int tz, int lp, int l, double pp,
                                             double p, const double *I1, const double *I2, const double *I3,
                                             double R, double *tv)
{
    double u[kYukTerms];
#pragma unroll
    for (int k = 0; k < kYukTerms; ++k) u[k] = 0.0;
    const bool diag = (lp == l);
    if (diag) {
        u[0] = I1[l];
        u[1] = (2.0 * s * (s + 1.0) - 3.0) * I1[l];
        u[2] = I2[l];
        double ilm1 = (l >= 1) ? I2[l - 1] : 0.0;
        u[3] = ls_factor(s, J, l) * pp * p * (I2[l + 1] - ilm1) / (2.0 * l + 1.0);
    }
    u[4] = s12_factor(s, J, lp, l) * I3[(l + lp) / 2];
    if (diag && l == 0 && s == 0) { u[5] = 1.0; u[7] = p * p + pp * pp; }
    if (diag && l == 0 && s == 1) { u[6] = 1.0; u[8] = p * p + pp * pp; }
    if (diag && l == 1 && s == 1 && J == 0) u[9] = pp * p;
    if (diag && l == 1 && s == 0 && J == 1) u[10] = pp * p;
    if (diag && l == 1 && s == 1 && J == 1) u[11] = pp * p;
    if (diag && l == 1 && s == 1 && J == 2) u[12] = pp * p;
    if (s == 1 && J == 1 && lp == 2 && l == 0) u[13] = pp * pp;
    if (s == 1 && J == 1 && lp == 0 && l == 2) u[13] = p * p;
    double v0 = 0.0;
#pragma unroll
    for (int k = 0; k < kYukTerms; ++k) {
        u[k] *= R;
        v0 = fma(gp[4 + k], u[k], v0);
    }
    if (s == 0 && l == 0 && lp == 0 && tz != 0) v0 += gp[18] * R;
    tv[0] = v0;
#pragma unroll
    for (int k = 0; k < kYukTerms; ++k)
        if (k + 1 < kMaxTerms) tv[k + 1] = u[k];
}

// Term values tv[0..kMaxTerms) of channel (s, J, tz) between the l-blocks lp
// (row, momentum pp) and l (column, momentum p): tv[0] = V0, tv[1..14] = u_a
// for the Yukawa set; tv[0] = V for Yamaguchi.  The angle integrals come from
// yukawa_angle_integrals (unused for Yamaguchi).
template <int GEN>
__device__ __forceinline__ void potential_terms(const double *gp, int s, int J, int tz, int lp, int l, double pp,
                                                double p, const double *I1, const double *I2, const double *I3,
                                                double R, double *tv)
{
#pragma unroll
    for (int t = 0; t < kMaxTerms; ++t) tv[t] = 0.0;
    if (GEN == WPCD_GEN_YAMAGUCHI) {
        if (lp == 0 && l == 0) tv[0] = gp[0] / ((pp * pp + gp[1] * gp[1]) * (p * p + gp[1] * gp[1]));
    } else {
        yukawa_terms(gp, s, J, tz, lp, l, pp, p, I1, I2, I3, R, tv);
    }
}

}  // namespace wpcd
