/*
 * wpcd_oracle.c -- plain, slow, FP64 CPU oracle for the wave-packet continuum
 * discretisation (WPCD) of the nucleon-nucleon Lippmann-Schwinger equation
 * (Miller, Ekstrom, Forssen, arXiv:2106.00454).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or constant with the CUDA
 * library: every constant and formula below is restated here from the paper.
 *
 * Every function follows the paper's steps in its own order and notation, with
 * no blocking or fusion: Sec. 3.2 (five-step WPCD recipe), App. A (S-matrix,
 * Stapp parametrisation, total cross section), App. B (resolvent in the
 * scattering-wave-packet basis), Sec. 2.1 (matrix-inversion method, used here
 * as an independent cross-check).  Where the paper is garbled the reading
 * taken is stated at the function; the same list is kept in the design notes.
 *
 * Units: momenta in fm^-1, energies in fm^-1 (E = k^2 / (2 mu)), potentials in
 * fm^2, with the partial-wave normalisation <k'|k> = delta(k'-k)/(k'k) of
 * Sec. 2, so that T = V + int k^2 dk V 2mu/(p^2 - k^2 + i0) T (no 2/pi).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- constants (reading G17: nonrelativistic kinematics, p^2 = m_N T_lab / 2) */
#define OR_HBARC 197.3269804     /* MeV fm */
#define OR_MN 938.918309         /* MeV, 2 m_p m_n / (m_p + m_n) */
#define OR_PI 3.14159265358979323846

double or_mu(void) { return 0.5 * OR_MN / OR_HBARC; } /* reduced mass, fm^-1 */
double or_hbarc(void) { return OR_HBARC; }
double or_mn(void) { return OR_MN; }

/* c.m. momentum (fm^-1) for a lab kinetic energy in MeV. */
double or_p_of_tlab(double tlab_mev) { return sqrt(OR_MN * tlab_mev / 2.0) / OR_HBARC; }

int or_version(void) { return 1; }

/* ------------------------------------------------------------------------- */
/* Gauss-Legendre rule on [-1,1] by Newton iteration on P_n (textbook).       */
/* ------------------------------------------------------------------------- */
int or_gauss_legendre(int n, double *x, double *w)
{
    if (n < 1) return -1;
    int m = (n + 1) / 2;
    for (int i = 0; i < m; ++i) {
        double z = cos(OR_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            /* P_n(z) and P_{n-1}(z) by the three-term recurrence */
            double pm1 = 1.0, pcur = z;
            for (int j = 2; j <= n; ++j) {
                double pnext = ((2.0 * j - 1.0) * z * pcur - (j - 1.0) * pm1) / j;
                pm1 = pcur;
                pcur = pnext;
            }
            dp = n * (z * pcur - pm1) / (z * z - 1.0);
            double dz = pcur / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double pm1 = 1.0, pcur = z;
        for (int j = 2; j <= n; ++j) {
            double pnext = ((2.0 * j - 1.0) * z * pcur - (j - 1.0) * pm1) / j;
            pm1 = pcur;
            pcur = pnext;
        }
        dp = n * (z * pcur - pm1) / (z * z - 1.0);
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        w[n - 1 - i] = w[i];
    }
    if (n % 2 == 1) x[m - 1] = 0.0;
    return 0;
}

/* Legendre polynomials P_0..P_L at x (three-term recurrence). */
static void legendre_all(int L, double x, double *P)
{
    P[0] = 1.0;
    if (L >= 1) P[1] = x;
    for (int l = 2; l <= L; ++l) P[l] = ((2.0 * l - 1.0) * x * P[l - 1] - (l - 1.0) * P[l - 2]) / l;
}

/* ------------------------------------------------------------------------- */
/* Step 1 of Sec. 3.2: free-wave-packet bin boundaries.                       */
/*   kind 0: tan^t map on a uniform angle grid, capped so that k_N = kmax     */
/*           (reading G2: the paper's Chebyshev/tan^t distribution made to    */
/*           end at a finite momentum);                                       */
/*   kind 1: the paper's Chebyshev distribution y_j = alpha tan^t((2j-1)pi/   */
/*           (4N)), y_0 = 0, unbounded above.                                 */
/* Within each bin Q Gauss-Legendre points give the fine quadrature of the    */
/* bin integrals of Eq. "WP potential matrix identity" (Sec. 3.2).            */
/* ------------------------------------------------------------------------- */
int or_mesh(int N, int kind, double alpha, double t, double kmax, int Q,
            double *kb, double *kq, double *wq)
{
    if (N < 2 || Q < 1) return -1;
    kb[0] = 0.0;
    if (kind == 0) {
        double thmax = atan(pow(kmax / alpha, 1.0 / t));
        for (int j = 1; j <= N; ++j) kb[j] = alpha * pow(tan(j * thmax / N), t);
        kb[N] = kmax;
    } else if (kind == 1) {
        for (int j = 1; j <= N; ++j) kb[j] = alpha * pow(tan((2.0 * j - 1.0) * OR_PI / (4.0 * N)), t);
    } else {
        return -1;
    }
    double *xg = (double *)malloc(sizeof(double) * Q), *wg = (double *)malloc(sizeof(double) * Q);
    or_gauss_legendre(Q, xg, wg);
    for (int i = 0; i < N; ++i) {
        double a = kb[i], b = kb[i + 1];
        for (int q = 0; q < Q; ++q) {
            kq[i * Q + q] = 0.5 * (a + b) + 0.5 * (b - a) * xg[q];
            wq[i * Q + q] = 0.5 * (b - a) * wg[q];
        }
    }
    free(xg);
    free(wg);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Potentials (inputs of the method, Sec. 2: partial-wave v^{sJ}_{l'l}(q',q)). */
/* ------------------------------------------------------------------------- */
typedef struct { int s, J, l, lp, coupled, tz; } or_channel;

/* generator 0: rank-1 Yamaguchi potential, params {lambda, beta}. */
/* generator 1: synthetic regulated Yukawa + contact set, params:
 *   [0..2] masses m1, m2, m3 (fm^-1), [3] regulator cutoff Lambda (fm^-1),
 *   [4..17] strengths of the 14 unit terms that form V0, [18] extra LO
 *   contact added to V0 in 1S0 channels with tz != 0.                      */
#define OR_NTERM_YUK 14

static double ls_factor(int s, int J, int l) { return 0.5 * (J * (J + 1.0) - l * (l + 1.0) - s * (s + 1.0)); }

/* tensor operator S12 in the |l s J> basis for s = 1 (standard LSJ values) */
static double s12_factor(int s, int J, int lp, int l)
{
    if (s != 1) return 0.0;
    if (lp == l) {
        if (l == J) return 2.0;
        if (l == J - 1) return -2.0 * (J - 1.0) / (2.0 * J + 1.0);
        if (l == J + 1) return -2.0 * (J + 2.0) / (2.0 * J + 1.0);
        return 0.0;
    }
    if ((lp == J - 1 && l == J + 1) || (lp == J + 1 && l == J - 1))
        return 6.0 * sqrt(J * (J + 1.0)) / (2.0 * J + 1.0);
    return 0.0;
}

/* 2 pi int_{-1}^{1} dx P_L(x) / (p'^2 + p^2 - 2 p' p x + m^2), 96-point GL, L = 0..Lmax */
typedef struct { int n; double x[96], w[96]; } or_angle_rule;

static void angle_integrals(const or_angle_rule *ar, double pp, double p, double m, int Lmax, double *Iout)
{
    double P[32];
    for (int L = 0; L <= Lmax; ++L) Iout[L] = 0.0;
    for (int ix = 0; ix < ar->n; ++ix) {
        double x = ar->x[ix];
        double F = 1.0 / (pp * pp + p * p - 2.0 * pp * p * x + m * m);
        legendre_all(Lmax, x, P);
        for (int L = 0; L <= Lmax; ++L) Iout[L] += ar->w[ix] * P[L] * F;
    }
    for (int L = 0; L <= Lmax; ++L) Iout[L] *= 2.0 * OR_PI;
}

/* The 14 unit terms of generator 1 in block (lp, l) of channel ch at (p', p).
 * out[a-1] for a = 1..14, regulated by exp(-(p'^2+p^2)/Lambda^2). */
static void yuk_terms(const or_angle_rule *ar, const double *gp, or_channel ch, int lp, int l,
                      double pp, double p, double *out)
{
    const double m1 = gp[0], m2 = gp[1], m3 = gp[2], Lam = gp[3];
    int s = ch.s, J = ch.J;
    int Lmax = J + 2;
    double I1[32], I2[32], I3[32];
    angle_integrals(ar, pp, p, m1, Lmax, I1);
    angle_integrals(ar, pp, p, m2, Lmax, I2);
    angle_integrals(ar, pp, p, m3, Lmax, I3);
    for (int a = 0; a < OR_NTERM_YUK; ++a) out[a] = 0.0;
    int diag = (lp == l);
    if (diag) {
        out[0] = I1[l];                                        /* central, m1 */
        out[1] = (2.0 * s * (s + 1.0) - 3.0) * I1[l];          /* spin-spin, m1 */
        out[2] = I2[l];                                        /* central, m2 */
        double Ilm1 = (l >= 1) ? I2[l - 1] : 0.0;              /* spin-orbit, m2 */
        out[3] = ls_factor(s, J, l) * pp * p * (I2[l + 1] - Ilm1) / (2.0 * l + 1.0);
    }
    out[4] = s12_factor(s, J, lp, l) * I3[(l + lp) / 2];       /* tensor, m3 */
    /* partial-wave contacts */
    if (diag && l == 0 && s == 0) { out[5] = 1.0; out[7] = p * p + pp * pp; }
    if (diag && l == 0 && s == 1) { out[6] = 1.0; out[8] = p * p + pp * pp; }
    if (diag && l == 1 && s == 1 && J == 0) out[9] = pp * p;
    if (diag && l == 1 && s == 0 && J == 1) out[10] = pp * p;
    if (diag && l == 1 && s == 1 && J == 1) out[11] = pp * p;
    if (diag && l == 1 && s == 1 && J == 2) out[12] = pp * p;
    if (s == 1 && J == 1 && lp == 2 && l == 0) out[13] = pp * pp;
    if (s == 1 && J == 1 && lp == 0 && l == 2) out[13] = p * p;
    double R = exp(-(pp * pp + p * p) / (Lam * Lam));
    for (int a = 0; a < OR_NTERM_YUK; ++a) out[a] *= R;
}

/* 96-point angle rule, filled once when the library is loaded. */
static or_angle_rule g_angle;
__attribute__((constructor)) static void or_init_angle_rule(void)
{
    g_angle.n = 96;
    or_gauss_legendre(96, g_angle.x, g_angle.w);
}

/* All potential terms t = 0..n_terms-1 (0 = V0, 1.. = unit terms) in block
 * (lp, l) of channel ch at momenta (p' = row, p = column). */
static void potential_terms(int gen, const double *gp, or_channel ch, int lp, int l, double pp, double p,
                            int n_terms, double *out)
{
    for (int t = 0; t < n_terms; ++t) out[t] = 0.0;
    if (gen == 0) {
        if (lp == 0 && l == 0) out[0] = gp[0] / ((pp * pp + gp[1] * gp[1]) * (p * p + gp[1] * gp[1]));
        return;
    }
    if (gen == 1) {
        double t[OR_NTERM_YUK];
        yuk_terms(&g_angle, gp, ch, lp, l, pp, p, t);
        double v0 = 0.0;
        for (int a = 0; a < OR_NTERM_YUK; ++a) v0 += gp[4 + a] * t[a];
        if (ch.s == 0 && l == 0 && lp == 0 && ch.tz != 0) v0 += gp[18] * exp(-(pp * pp + p * p) / (gp[3] * gp[3]));
        out[0] = v0;
        for (int a = 1; a < n_terms && a <= OR_NTERM_YUK; ++a) out[a] = t[a - 1];
    }
}

double or_potential(int gen, const double *gp, int ch_s, int ch_J, int ch_l, int ch_lp, int ch_coupled,
                    int ch_tz, int lp, int l, int term, double pp, double p)
{
    or_channel ch = {ch_s, ch_J, ch_l, ch_lp, ch_coupled, ch_tz};
    double out[OR_NTERM_YUK + 1];
    potential_terms(gen, gp, ch, lp, l, pp, p, OR_NTERM_YUK + 1, out);
    return (term >= 0 && term <= OR_NTERM_YUK) ? out[term] : 0.0;
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.1: weighting function f(k) and norm N_i of a free wave packet       */
/* (Eq. "definition free wave-packet").  Reading G1: momentum packets have    */
/* f = 1, N_i = dk_i; energy packets f = sqrt(k/mu), N_i = dE_i (this is the  */
/* pairing that makes <x_i|x_i> = 1).                                         */
/* ------------------------------------------------------------------------- */
static double wp_f(int wp_kind, double k) { return wp_kind == 0 ? 1.0 : sqrt(k / or_mu()); }
static double wp_norm(int wp_kind, double ka, double kb)
{
    if (wp_kind == 0) return kb - ka;
    return (kb * kb - ka * ka) / (2.0 * or_mu());
}

/* H0_ii = <x_i|h0|x_i> = (1/N_i) int_{D_i} dk f(k)^2 k^2/(2 mu)  (reading G15:
 * the exact matrix element instead of the bin-midpoint approximation). */
double or_h0(int wp_kind, double ka, double kb)
{
    double mu = or_mu();
    if (wp_kind == 0) return (kb * kb * kb - ka * ka * ka) / (3.0 * (kb - ka)) / (2.0 * mu);
    double Ea = ka * ka / (2.0 * mu), Eb = kb * kb / (2.0 * mu);
    return 0.5 * (Ea + Eb);
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.2, Eq. "WP potential matrix identity": bin-averaged potential       */
/*   V_ij = (N_i N_j)^-1/2 int_{D_i} int_{D_j} k'k dk'dk f(k')f(k) v(k',k)    */
/* evaluated with the Q-point rule of each bin.  The matrix of one channel is */
/* n x n, n = K N, with l-blocks (K = 2 for coupled channels, block 0 =       */
/* l = J-1, block 1 = l = J+1, each on the same degenerate FWP basis).        */
/* Vt: [n_terms][n][n] row-major.                                             */
/* ------------------------------------------------------------------------- */
int or_project_channel(int N, const double *kb, int Q, const double *kq, const double *wq, int wp_kind,
                       int ch_s, int ch_J, int ch_l, int ch_lp, int ch_coupled, int ch_tz,
                       int gen, const double *gp, int n_terms, double *Vt)
{
    int K = ch_coupled ? 2 : 1;
    int n = K * N;
    int NQ = N * Q;
    int lblk[2];
    if (ch_coupled) { lblk[0] = ch_J - 1; lblk[1] = ch_J + 1; }
    else { lblk[0] = ch_l; lblk[1] = ch_l; }
    /* fine-point weights omega_a = w_a k_a f(k_a) / sqrt(N_i) */
    double *om = (double *)malloc(sizeof(double) * NQ);
    for (int i = 0; i < N; ++i) {
        double Ni = wp_norm(wp_kind, kb[i], kb[i + 1]);
        for (int q = 0; q < Q; ++q) {
            int a = i * Q + q;
            om[a] = wq[a] * kq[a] * wp_f(wp_kind, kq[a]) / sqrt(Ni);
        }
    }
    or_channel ch = {ch_s, ch_J, ch_l, ch_lp, ch_coupled, ch_tz};
    memset(Vt, 0, sizeof(double) * (size_t)n_terms * n * n);
    for (int al = 0; al < K; ++al)
        for (int be = 0; be < K; ++be) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic)
#endif
            for (int i = 0; i < N; ++i)
                for (int j = 0; j < N; ++j) {
                    double acc[OR_NTERM_YUK + 1], v[OR_NTERM_YUK + 1];
                    for (int t = 0; t < n_terms; ++t) acc[t] = 0.0;
                    for (int qa = 0; qa < Q; ++qa)
                        for (int qb = 0; qb < Q; ++qb) {
                            int a = i * Q + qa, b = j * Q + qb;
                            potential_terms(gen, gp, ch, lblk[al], lblk[be], kq[a], kq[b], n_terms, v);
                            for (int t = 0; t < n_terms; ++t) acc[t] += om[a] * om[b] * v[t];
                        }
                    for (int t = 0; t < n_terms; ++t)
                        Vt[(size_t)t * n * n + (size_t)(al * N + i) * n + (be * N + j)] = acc[t];
                }
        }
    free(om);
    return 0;
}

/* Same bin reduction applied to caller-supplied fine-grid values
 * vfine[(al*NQ + a)*(K*NQ) + (be*NQ + b)] of one term. */
int or_project_fine(int N, const double *kb, int Q, const double *kq, const double *wq, int wp_kind, int K,
                    const double *vfine, double *V)
{
    int n = K * N, NQ = N * Q;
    double *om = (double *)malloc(sizeof(double) * NQ);
    for (int i = 0; i < N; ++i) {
        double Ni = wp_norm(wp_kind, kb[i], kb[i + 1]);
        for (int q = 0; q < Q; ++q) {
            int a = i * Q + q;
            om[a] = wq[a] * kq[a] * wp_f(wp_kind, kq[a]) / sqrt(Ni);
        }
    }
    for (int al = 0; al < K; ++al)
        for (int be = 0; be < K; ++be)
            for (int i = 0; i < N; ++i)
                for (int j = 0; j < N; ++j) {
                    double acc = 0.0;
                    for (int qa = 0; qa < Q; ++qa)
                        for (int qb = 0; qb < Q; ++qb) {
                            int a = i * Q + qa, b = j * Q + qb;
                            acc += om[a] * om[b] * vfine[(size_t)(al * NQ + a) * (K * NQ) + (be * NQ + b)];
                        }
                    V[(size_t)(al * N + i) * n + (be * N + j)] = acc;
                }
    free(om);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Step 2 of Sec. 3.2: diagonalise H = C D C^T.  Cyclic-by-row two-sided      */
/* Jacobi (Golub & Van Loan, cited in Sec. 4.2.2).  Eigenvalues ascending,    */
/* eigenvectors in the columns of C (row-major C[i*n + s]), each with its     */
/* largest-magnitude component made positive.  Returns the sweep count, or    */
/* -1 if off(A) did not fall below 1e-15 ||A||_F within 30 sweeps.           */
/* ------------------------------------------------------------------------- */
int or_jacobi(int n, const double *H, double *eps, double *C)
{
    double *A = (double *)malloc(sizeof(double) * n * n);
    memcpy(A, H, sizeof(double) * n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) C[i * n + j] = (i == j) ? 1.0 : 0.0;
    double fro = 0.0;
    for (int i = 0; i < n * n; ++i) fro += A[i] * A[i];
    fro = sqrt(fro);
    int sweeps = 0, converged = 0;
    for (; sweeps <= 30; ++sweeps) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                if (i != j) off += A[i * n + j] * A[i * n + j];
        if (sqrt(off) <= 1e-15 * fro) { converged = 1; break; }
        if (sweeps == 30) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                /* symmetric 2x2 Schur decomposition */
                double tau = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                double t = (tau >= 0.0) ? 1.0 / (tau + sqrt(1.0 + tau * tau))
                                        : -1.0 / (-tau + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                /* A <- A J (columns p, q) */
                for (int k = 0; k < n; ++k) {
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                /* A <- J^T A (rows p, q) */
                for (int k = 0; k < n; ++k) {
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                A[p * n + q] = 0.0; /* zero by construction of the rotation */
                A[q * n + p] = 0.0;
                /* C <- C J */
                for (int k = 0; k < n; ++k) {
                    double vkp = C[k * n + p], vkq = C[k * n + q];
                    C[k * n + p] = c * vkp - s * vkq;
                    C[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < n; ++i) eps[i] = A[i * n + i];
    /* sort ascending (selection sort, permuting columns of C) */
    for (int i = 0; i < n - 1; ++i) {
        int kmin = i;
        for (int j = i + 1; j < n; ++j)
            if (eps[j] < eps[kmin]) kmin = j;
        if (kmin != i) {
            double tmp = eps[i]; eps[i] = eps[kmin]; eps[kmin] = tmp;
            for (int r = 0; r < n; ++r) {
                double c2 = C[r * n + i]; C[r * n + i] = C[r * n + kmin]; C[r * n + kmin] = c2;
            }
        }
    }
    for (int s = 0; s < n; ++s) {
        int imax = 0;
        for (int r = 1; r < n; ++r)
            if (fabs(C[r * n + s]) > fabs(C[imax * n + s])) imax = r;
        if (C[imax * n + s] < 0.0)
            for (int r = 0; r < n; ++r) C[r * n + s] = -C[r * n + s];
    }
    free(A);
    return converged ? sweeps : -1;
}

/* ------------------------------------------------------------------------- */
/* Step 3 of Sec. 3.2, Eq. "pseudostate wave packet boundaries": SWP bin      */
/* boundaries from the positive eigenvalues e_1 < ... < e_m of one branch:    */
/*   B_1 = 0, B_i = (e_{i-1} + e_i)/2, B_{m+1} = e_m + (B_m - B_{m-1})/2.     */
/* Coupled channels (Sec. 3.1, K = 2): reading G14 -- the positive            */
/* eigenvalues, sorted ascending, are dealt alternately to the two branches   */
/* starting from the top (largest -> branch 1 of 0/1, next -> branch 0, ...). */
/* Output: branch[s] (-1 for a bound state), pos[s] = index of s inside its   */
/* branch, and per branch its boundary array bnd[b*(n+1) + 0..m_b].           */
/* Returns the number of bound states.                                        */
/* ------------------------------------------------------------------------- */
int or_swp_boundaries(int n, int K, const double *eps, int *branch, int *pos, int *mcount, double *bnd)
{
    int nb = 0;
    while (nb < n && eps[nb] < 0.0) ++nb;
    for (int s = 0; s < nb; ++s) { branch[s] = -1; pos[s] = -1; }
    mcount[0] = mcount[1] = 0;
    int npos = n - nb;
    for (int r = 0; r < npos; ++r) {
        int s = n - 1 - r; /* r-th from the top */
        int b = (K == 2) ? ((r % 2 == 0) ? 1 : 0) : 0;
        branch[s] = b;
    }
    /* positions inside each branch, ascending */
    for (int s = nb; s < n; ++s) {
        int b = branch[s];
        pos[s] = mcount[b]++;
    }
    for (int b = 0; b < K; ++b) {
        int m = mcount[b];
        double *B = bnd + (size_t)b * (n + 1);
        double *e = (double *)malloc(sizeof(double) * (m > 0 ? m : 1));
        int c = 0;
        for (int s = nb; s < n; ++s)
            if (branch[s] == b) e[c++] = eps[s];
        if (m >= 2) {
            B[0] = 0.0;
            for (int i = 1; i < m; ++i) B[i] = 0.5 * (e[i - 1] + e[i]);
            B[m] = e[m - 1] + 0.5 * (B[m - 1] - B[m - 2]);
        }
        free(e);
    }
    return nb;
}

/* ------------------------------------------------------------------------- */
/* Step 4 of Sec. 3.2 and App. B: the resolvent of the full Hamiltonian in    */
/* the SWP basis, averaged over the on-shell energy.                          */
/* Point resolvent (App. B, with reading G6 for the printed log ratio):       */
/*   <z_s|g(E)|z_s> = [ln|(E - B_s)/(E - B_{s+1})| - i pi 1{E in [B_s,        */
/*   B_{s+1}]}] / dB_s.                                                       */
/* Energy average over the free bin [Ea, Eb] containing E (reading G8; the    */
/* domain of Eq. "resolvent energy averaging"), written with                  */
/* X(a, b) = (a - b) ln|a - b| (the App. B closed form W with reading G7 for  */
/* its overall sign):                                                         */
/*   gbar = [X(Eb,B_s) - X(Ea,B_s) - X(Eb,B_{s+1}) + X(Ea,B_{s+1})]/(dE dB)   */
/*          - i pi |[Ea,Eb] ^ [B_s,B_{s+1}]| / (dE dB).                       */
/* A bound state e_b < 0 (second line of Eq. "LS equation in WP basis") gets  */
/* its 1/(E - e_b) averaged the same way (reading G20):                       */
/*   ln((Eb - e_b)/(Ea - e_b)) / dE.                                          */
/* ------------------------------------------------------------------------- */
static double xlogabs(double d) { return (d == 0.0) ? 0.0 : d * log(fabs(d)); }

void or_gbar_scatt(double Ea, double Eb, double Bs, double Bs1, double *re, double *im)
{
    double dE = Eb - Ea, dB = Bs1 - Bs;
    double num = xlogabs(Eb - Bs) - xlogabs(Ea - Bs) - xlogabs(Eb - Bs1) + xlogabs(Ea - Bs1);
    *re = num / (dE * dB);
    double lo = (Ea > Bs) ? Ea : Bs, hi = (Eb < Bs1) ? Eb : Bs1;
    double ov = (hi > lo) ? hi - lo : 0.0;
    *im = -OR_PI * ov / (dE * dB);
}

double or_gbar_bound(double Ea, double Eb, double eb) { return log((Eb - eb) / (Ea - eb)) / (Eb - Ea); }

/* Point resolvent (for tests of the average). */
void or_g_point(double E, double Bs, double Bs1, double *re, double *im)
{
    double dB = Bs1 - Bs;
    *re = log(fabs((E - Bs) / (E - Bs1))) / dB;
    *im = (E >= Bs && E <= Bs1) ? -OR_PI / dB : 0.0;
}

/* ------------------------------------------------------------------------- */
/* Step 5 of Sec. 3.2, Eq. "on-shell T-mat element in fWP" with the sums of   */
/* Eq. "LS equation in WP basis" (reading G12: the sum runs over every        */
/* eigenstate s, bound and scattering, and over both l-blocks):               */
/*   T_{a b}(i) = V_{(a,i),(b,i)} + sum_s (VC)_{(a,i),s} g_s (VC)_{(b,i),s}.  */
/* The contraction with a given diagonal g (complex) is split out so that it  */
/* can be checked on its own against the spectral identity.                   */
/* R: rows of VC for the K rows (a,i), R[a*n + s].                            */
/* ------------------------------------------------------------------------- */
void or_contract(int n, int K, const double *Vdiag /*K*K*/, const double *R, const double *g_re,
                 const double *g_im, double *T_re, double *T_im)
{
    for (int a = 0; a < K; ++a)
        for (int b = 0; b < K; ++b) {
            double tr = Vdiag[a * K + b], ti = 0.0;
            for (int s = 0; s < n; ++s) {
                double rr = R[a * n + s] * R[b * n + s];
                tr += rr * g_re[s];
                ti += rr * g_im[s];
            }
            T_re[a * K + b] = tr;
            T_im[a * K + b] = ti;
        }
}

/* ------------------------------------------------------------------------- */
/* App. A: S = 1 - 2 pi i T with the density of states of the Sec. 2         */
/* normalisation (reading G4): S = 1 - 2 pi i mu p T(p,p).  T in the          */
/* continuum basis is obtained from the packet basis by Eq. "operator in cont */
/* and disc representation" at q = the bin midpoint (Sec. 3.2, last para,     */
/* reading G18).  Phase shifts: uncoupled delta = arg(S)/2; coupled channels  */
/* in the Stapp parametrisation, delta_-+ = arg(S_11/22)/2 and                */
/* eps_J = asin(Re[-i S_12 exp(-i(delta_- + delta_+))])/2.                    */
/* Angles in degrees.  out: {delta or delta_-, delta_+, eps_J}.               */
/* ------------------------------------------------------------------------- */
void or_phases_from_S(int K, const double complex *S, double *out)
{
    const double deg = 180.0 / OR_PI;
    if (K == 1) {
        out[0] = 0.5 * carg(S[0]) * deg;
        out[1] = 0.0;
        out[2] = 0.0;
        return;
    }
    double dm = 0.5 * carg(S[0]), dp = 0.5 * carg(S[3]);
    double complex z = -I * S[1] * cexp(-I * (dm + dp));
    double x = creal(z);
    if (x > 1.0) x = 1.0;
    if (x < -1.0) x = -1.0;
    out[0] = dm * deg;
    out[1] = dp * deg;
    out[2] = 0.5 * asin(x) * deg;
}

void or_S_from_T(int K, double p, const double complex *T, double complex *S)
{
    double mu = or_mu();
    for (int a = 0; a < K; ++a)
        for (int b = 0; b < K; ++b)
            S[a * K + b] = ((a == b) ? 1.0 : 0.0) - 2.0 * OR_PI * I * mu * p * T[a * K + b];
}

/* ------------------------------------------------------------------------- */
/* One channel-solve (Sec. 3.2 steps 2-5 for every free bin i = 0..N-1):     */
/*   H = diag(H0) (per l-block) + Vt[0] + sum_a c_a Vt[a];                    */
/*   eigenpairs; SWP boundaries; gbar for free bin i; T_ii; continuum T at    */
/*   q = kbar_i; S; phases.                                                   */
/* mode 0: resolvent averaged over free bin i (reading G8); mode 1: over SWP  */
/* bin i (the printed App. B form; uncoupled channels without bound states). */
/* Outputs: Tc [N][K][K] complex continuum T(kbar_i,kbar_i) in fm^2,          */
/*          ph [N][3] degrees, eps [n].  Returns the number of bound states,  */
/*          or a negative code (-1 no convergence, -2 bad branch sizes,       */
/*          -4 mode 1 on a coupled channel or with a bound state).            */
/* ------------------------------------------------------------------------- */
/* Sec. 5.1.1, Eq. "interpolation point": the point of free bin i (boundaries */
/* k_i < k_{i+1}) at which its T is converted to the continuum and its phase  */
/* placed for the interpolation, q = k_i + (n/m)(k_{i+1} - k_i), written as   */
/* the weighted average (1 - f) k_i + f k_{i+1} with f = n/m; f = 1/2 is the  */
/* bin midpoint (0.5 k_i + 0.5 k_{i+1} is then exactly 0.5 (k_i + k_{i+1})).  */
static double ip_point(const double *kb, int i, double f) { return (1.0 - f) * kb[i] + f * kb[i + 1]; }

int or_channel_solve_ip(int N, const double *kb, int wp_kind, int K, int n_terms, const double *Vt,
                        const double *c, int mode, double frac, double complex *Tc, double *ph, double *eps_out,
                        int *sweeps_out);

int or_channel_solve(int N, const double *kb, int wp_kind, int K, int n_terms, const double *Vt,
                     const double *c, int mode, double complex *Tc, double *ph, double *eps_out, int *sweeps_out)
{
    return or_channel_solve_ip(N, kb, wp_kind, K, n_terms, Vt, c, mode, 0.5, Tc, ph, eps_out, sweeps_out);
}

/* or_channel_solve with the conversion point of each bin at fraction frac of */
/* the bin (0 < frac < 1; 0.5 = the midpoint of reading G18).                 */
int or_channel_solve_ip(int N, const double *kb, int wp_kind, int K, int n_terms, const double *Vt,
                        const double *c, int mode, double frac, double complex *Tc, double *ph, double *eps_out,
                        int *sweeps_out)
{
    int n = K * N;
    double mu = or_mu();
    double *H = (double *)malloc(sizeof(double) * n * n);
    double *V = (double *)malloc(sizeof(double) * n * n);
    double *C = (double *)malloc(sizeof(double) * n * n);
    double *eps = (double *)malloc(sizeof(double) * n);
    for (int i = 0; i < n * n; ++i) {
        double v = Vt[i];
        for (int a = 1; a < n_terms; ++a) v += c[a - 1] * Vt[(size_t)a * n * n + i];
        V[i] = v;
        H[i] = v;
    }
    for (int blk = 0; blk < K; ++blk)
        for (int i = 0; i < N; ++i) H[(blk * N + i) * n + (blk * N + i)] += or_h0(wp_kind, kb[i], kb[i + 1]);
    int sw = or_jacobi(n, H, eps, C);
    if (sweeps_out) *sweeps_out = sw;
    int rc = 0;
    if (sw < 0) rc = -1;
    int *branch = (int *)malloc(sizeof(int) * n), *pos = (int *)malloc(sizeof(int) * n);
    int mcount[2];
    double *bnd = (double *)malloc(sizeof(double) * 2 * (n + 1));
    int nb = or_swp_boundaries(n, K, eps, branch, pos, mcount, bnd);
    for (int b = 0; b < K; ++b)
        if (mcount[b] < 2) rc = -2;
    /* SWP-index averaging (App. B as printed, reading G8 alternative): the      */
    /* average runs over SWP bin i of the one branch, which lines up with free   */
    /* bin i only for an uncoupled channel without bound states.                  */
    if (mode == 1 && rc == 0 && (K != 1 || nb != 0)) rc = -4;
    double *R = (double *)malloc(sizeof(double) * K * n);
    double *gre = (double *)malloc(sizeof(double) * n), *gim = (double *)malloc(sizeof(double) * n);
    for (int i = 0; i < N && rc == 0; ++i) {
        double Ea = kb[i] * kb[i] / (2.0 * mu), Eb = kb[i + 1] * kb[i + 1] / (2.0 * mu);
        if (mode == 1) { /* average over SWP bin i instead of free bin i */
            Ea = bnd[i];
            Eb = bnd[i + 1];
        }
        /* rows (a, i) of VC */
        for (int a = 0; a < K; ++a)
            for (int s = 0; s < n; ++s) {
                double acc = 0.0;
                for (int j = 0; j < n; ++j) acc += V[(a * N + i) * n + j] * C[j * n + s];
                R[a * n + s] = acc;
            }
        for (int s = 0; s < n; ++s) {
            if (branch[s] < 0) {
                gre[s] = or_gbar_bound(Ea, Eb, eps[s]);
                gim[s] = 0.0;
            } else {
                const double *B = bnd + (size_t)branch[s] * (n + 1);
                or_gbar_scatt(Ea, Eb, B[pos[s]], B[pos[s] + 1], &gre[s], &gim[s]);
            }
        }
        double Vd[4], Tr[4], Ti[4];
        for (int a = 0; a < K; ++a)
            for (int b = 0; b < K; ++b) Vd[a * K + b] = V[(a * N + i) * n + (b * N + i)];
        or_contract(n, K, Vd, R, gre, gim, Tr, Ti);
        /* continuum normalisation at q = kbar_i (the interpolation point of bin i) */
        double kbar = ip_point(kb, i, frac);
        double Ni = wp_norm(wp_kind, kb[i], kb[i + 1]);
        double fac = wp_f(wp_kind, kbar) * wp_f(wp_kind, kbar) / (Ni * kbar * kbar);
        double complex Tq[4], S[4];
        for (int ab = 0; ab < K * K; ++ab) {
            Tq[ab] = fac * (Tr[ab] + I * Ti[ab]);
            Tc[(size_t)i * K * K + ab] = Tq[ab];
        }
        or_S_from_T(K, kbar, Tq, S);
        or_phases_from_S(K, S, ph + 3 * i);
    }
    if (eps_out) memcpy(eps_out, eps, sizeof(double) * n);
    free(H); free(V); free(C); free(eps); free(branch); free(pos); free(bnd); free(R); free(gre); free(gim);
    return rc < 0 ? rc : nb;
}

/* ------------------------------------------------------------------------- */
/* Point-resolvent variant (App. B point form with reading G6): no energy     */
/* average; at each requested energy E = p^2/(2 mu), with i the free bin      */
/* holding p,                                                                 */
/*   T_ab(E) = V_(a,i),(b,i) + sum_s (VC)_(a,i),s g_s(E) (VC)_(b,i),s,        */
/*   g_s(E) = [ln|(E - B_s)/(E - B_{s+1})| - i pi 1{E in [B_s, B_{s+1}]}]/dB_s */
/*   for a scattering state, 1/(E - e_b) for a bound state,                   */
/* converted to the continuum at q = p itself (the pointwise reading of Eq.   */
/* "operator in cont and disc representation"); S and the phases at p, with   */
/* no interpolation.  p_list [nE] ascending inside the mesh.                  */
/* Outputs: Tc [nE][K][K] complex fm^2, ph [nE][3] degrees.  Returns the      */
/* number of bound states or a negative code (-1, -2 as above; -3 an energy   */
/* outside the mesh).                                                         */
/* ------------------------------------------------------------------------- */
int or_channel_solve_point(int N, const double *kb, int wp_kind, int K, int n_terms, const double *Vt,
                           const double *c, int nE, const double *p_list, double complex *Tc, double *ph)
{
    int n = K * N;
    double mu = or_mu();
    double *H = (double *)malloc(sizeof(double) * n * n);
    double *V = (double *)malloc(sizeof(double) * n * n);
    double *C = (double *)malloc(sizeof(double) * n * n);
    double *eps = (double *)malloc(sizeof(double) * n);
    for (int i = 0; i < n * n; ++i) {
        double v = Vt[i];
        for (int a = 1; a < n_terms; ++a) v += c[a - 1] * Vt[(size_t)a * n * n + i];
        V[i] = v;
        H[i] = v;
    }
    for (int blk = 0; blk < K; ++blk)
        for (int i = 0; i < N; ++i) H[(blk * N + i) * n + (blk * N + i)] += or_h0(wp_kind, kb[i], kb[i + 1]);
    int rc = or_jacobi(n, H, eps, C) < 0 ? -1 : 0;
    int *branch = (int *)malloc(sizeof(int) * n), *pos = (int *)malloc(sizeof(int) * n);
    int mcount[2];
    double *bnd = (double *)malloc(sizeof(double) * 2 * (n + 1));
    int nb = or_swp_boundaries(n, K, eps, branch, pos, mcount, bnd);
    for (int b = 0; b < K; ++b)
        if (mcount[b] < 2) rc = -2;
    double *R = (double *)malloc(sizeof(double) * K * n);
    double *gre = (double *)malloc(sizeof(double) * n), *gim = (double *)malloc(sizeof(double) * n);
    for (int e = 0; e < nE && rc == 0; ++e) {
        double p = p_list[e], E = p * p / (2.0 * mu);
        int i = -1;
        for (int j = 0; j < N; ++j)
            if (kb[j] <= p && p < kb[j + 1]) i = j;
        if (i < 0) {
            rc = -3;
            break;
        }
        for (int a = 0; a < K; ++a)
            for (int s2 = 0; s2 < n; ++s2) {
                double acc = 0.0;
                for (int j = 0; j < n; ++j) acc += V[(a * N + i) * n + j] * C[j * n + s2];
                R[a * n + s2] = acc;
            }
        for (int s2 = 0; s2 < n; ++s2) {
            if (branch[s2] < 0) {
                gre[s2] = 1.0 / (E - eps[s2]);
                gim[s2] = 0.0;
            } else {
                const double *B = bnd + (size_t)branch[s2] * (n + 1);
                or_g_point(E, B[pos[s2]], B[pos[s2] + 1], &gre[s2], &gim[s2]);
            }
        }
        double Vd[4], Tr[4], Ti[4];
        for (int a = 0; a < K; ++a)
            for (int b = 0; b < K; ++b) Vd[a * K + b] = V[(a * N + i) * n + (b * N + i)];
        or_contract(n, K, Vd, R, gre, gim, Tr, Ti);
        double Ni = wp_norm(wp_kind, kb[i], kb[i + 1]);
        double fac = wp_f(wp_kind, p) * wp_f(wp_kind, p) / (Ni * p * p);
        double complex Tq[4], S[4];
        for (int ab = 0; ab < K * K; ++ab) {
            Tq[ab] = fac * (Tr[ab] + I * Ti[ab]);
            Tc[(size_t)e * K * K + ab] = Tq[ab];
        }
        or_S_from_T(K, p, Tq, S);
        or_phases_from_S(K, S, ph + 3 * e);
    }
    free(H); free(V); free(C); free(eps); free(branch); free(pos); free(bnd); free(R); free(gre); free(gim);
    return rc < 0 ? rc : nb;
}

/* ------------------------------------------------------------------------- */
/* Sec. 5.1.1, Eq. "linear interpolation": phase shifts interpolated linearly */
/* in q between consecutive bin midpoints (reading G3: the segment joining    */
/* kbar_j and kbar_{j+1} with kbar_j <= p < kbar_{j+1}; the end segments are  */
/* extended below the first and above the last midpoint).  Before             */
/* interpolating, delta_{j+1} is moved by a multiple of 180 deg to lie within */
/* 90 deg of delta_j (reading G19); the result is mapped back to (-90, 90].   */
/* The mixing angle is interpolated as is.                                    */
/* ------------------------------------------------------------------------- */
static double wrap90(double d)
{
    while (d > 90.0) d -= 180.0;
    while (d <= -90.0) d += 180.0;
    return d;
}

void or_interp_phase_ip(int N, const double *kb, const double *ph /*[N][3]*/, int K, double p, double frac,
                        double *out);

void or_interp_phase(int N, const double *kb, const double *ph /*[N][3]*/, int K, double p, double *out)
{
    or_interp_phase_ip(N, kb, ph, K, p, 0.5, out);
}

/* The same between the interpolation points q_j = (1 - frac) k_j + frac k_{j+1} */
/* of consecutive bins (Eq. "interpolation point"; frac = 0.5: midpoints).      */
void or_interp_phase_ip(int N, const double *kb, const double *ph /*[N][3]*/, int K, double p, double frac,
                        double *out)
{
    int j = -1;
    for (int i = 0; i < N; ++i)
        if (ip_point(kb, i, frac) <= p) j = i;
    if (j < 0) j = 0;
    if (j > N - 2) j = N - 2;
    double q0 = ip_point(kb, j, frac), q1 = ip_point(kb, j + 1, frac);
    double w = (p - q0) / (q1 - q0);
    int ncomp = (K == 2) ? 2 : 1;
    for (int c = 0; c < ncomp; ++c) {
        double d0 = ph[3 * j + c], d1 = ph[3 * (j + 1) + c];
        double k = round((d0 - d1) / 180.0);
        d1 += 180.0 * k;
        out[c] = wrap90(d0 + w * (d1 - d0));
    }
    if (K == 2) {
        double e0 = ph[3 * j + 2], e1 = ph[3 * (j + 1) + 2];
        out[2] = e0 + w * (e1 - e0);
    } else {
        out[1] = 0.0;
        out[2] = 0.0;
    }
}

/* ------------------------------------------------------------------------- */
/* App. A: total cross section.  Reading G13: the optical theorem written as  */
/* the partial-wave sum for two spin-1/2 particles,                           */
/*   sigma = pi/(2 p^2) sum_channels (2J+1) sum_{l in channel} Re(1 - S_ll),  */
/* with S rebuilt from the interpolated Stapp parameters at the exact p.      */
/* Returns the channel's contribution (2J+1) sum_l Re(1 - S_ll).              */
/* ------------------------------------------------------------------------- */
double or_sigma_term(int J, int K, const double *phdeg)
{
    const double rad = OR_PI / 180.0;
    if (K == 1) return (2.0 * J + 1.0) * (1.0 - cos(2.0 * phdeg[0] * rad));
    double c2e = cos(2.0 * phdeg[2] * rad);
    return (2.0 * J + 1.0) * ((1.0 - c2e * cos(2.0 * phdeg[0] * rad)) + (1.0 - c2e * cos(2.0 * phdeg[1] * rad)));
}

double or_sigma_prefactor_mb(double p) { return OR_PI / (2.0 * p * p) * 10.0; } /* 1 fm^2 = 10 mb */

/* ------------------------------------------------------------------------- */
/* Sec. 2.1: matrix-inversion (MI) cross-check, real K-matrix with the        */
/* Haftel-Tabakin pole subtraction (reading G5 for the D vector):             */
/*   D_j = w_j k_j^2 2mu/(p^2 - k_j^2) (j <= NQ),                             */
/*   D_{NQ+1} = -2mu p^2 sum_j w_j/(p^2 - k_j^2),                             */
/*   (1 - V D) K = V on the grid {k_j} + {p};                                 */
/* grid k = c tan(pi (1+x)/4) over Gauss-Legendre x.  LU with partial         */
/* pivoting (own code).  Output: the on-shell K (K x K, fm^2).                */
/* ------------------------------------------------------------------------- */
static int lu_solve(int n, double *A, double *B, int nrhs)
{
    int *piv = (int *)malloc(sizeof(int) * n);
    for (int k = 0; k < n; ++k) {
        int pmax = k;
        for (int i = k + 1; i < n; ++i)
            if (fabs(A[i * n + k]) > fabs(A[pmax * n + k])) pmax = i;
        piv[k] = pmax;
        if (A[pmax * n + k] == 0.0) { free(piv); return -1; }
        if (pmax != k) {
            for (int j = 0; j < n; ++j) { double t = A[k * n + j]; A[k * n + j] = A[pmax * n + j]; A[pmax * n + j] = t; }
            for (int j = 0; j < nrhs; ++j) { double t = B[k * nrhs + j]; B[k * nrhs + j] = B[pmax * nrhs + j]; B[pmax * nrhs + j] = t; }
        }
        for (int i = k + 1; i < n; ++i) {
            double f = A[i * n + k] / A[k * n + k];
            A[i * n + k] = f;
            for (int j = k + 1; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
            for (int j = 0; j < nrhs; ++j) B[i * nrhs + j] -= f * B[k * nrhs + j];
        }
    }
    for (int j = 0; j < nrhs; ++j)
        for (int i = n - 1; i >= 0; --i) {
            double acc = B[i * nrhs + j];
            for (int k = i + 1; k < n; ++k) acc -= A[i * n + k] * B[k * nrhs + j];
            B[i * nrhs + j] = acc / A[i * n + i];
        }
    free(piv);
    return 0;
}

int or_mi_kmatrix(int gen, const double *gp, int ch_s, int ch_J, int ch_l, int ch_lp, int ch_coupled, int ch_tz,
                  int n_terms, const double *c, int NQ, double cmap, double p, double *Kout)
{
    int K = ch_coupled ? 2 : 1;
    int M = NQ + 1, n = K * M;
    double mu = or_mu();
    double *xg = (double *)malloc(sizeof(double) * NQ), *wg = (double *)malloc(sizeof(double) * NQ);
    double *k = (double *)malloc(sizeof(double) * M), *w = (double *)malloc(sizeof(double) * NQ);
    double *D = (double *)malloc(sizeof(double) * M);
    or_gauss_legendre(NQ, xg, wg);
    for (int j = 0; j < NQ; ++j) {
        double th = OR_PI * (1.0 + xg[j]) / 4.0;
        k[j] = cmap * tan(th);
        w[j] = cmap * (OR_PI / 4.0) * wg[j] / (cos(th) * cos(th));
    }
    k[NQ] = p;
    double sum = 0.0;
    for (int j = 0; j < NQ; ++j) {
        D[j] = w[j] * k[j] * k[j] * 2.0 * mu / (p * p - k[j] * k[j]);
        sum += w[j] / (p * p - k[j] * k[j]);
    }
    D[NQ] = -2.0 * mu * p * p * sum;
    int lblk[2];
    if (ch_coupled) { lblk[0] = ch_J - 1; lblk[1] = ch_J + 1; }
    else { lblk[0] = ch_l; lblk[1] = ch_l; }
    or_channel ch = {ch_s, ch_J, ch_l, ch_lp, ch_coupled, ch_tz};
    double *V = (double *)malloc(sizeof(double) * n * n);
    for (int al = 0; al < K; ++al)
        for (int be = 0; be < K; ++be)
            for (int i = 0; i < M; ++i)
                for (int j = 0; j < M; ++j) {
                    double vt[OR_NTERM_YUK + 1];
                    potential_terms(gen, gp, ch, lblk[al], lblk[be], k[i], k[j], n_terms, vt);
                    double v = vt[0];
                    for (int t = 1; t < n_terms; ++t) v += c[t - 1] * vt[t];
                    V[(al * M + i) * n + (be * M + j)] = v;
                }
    double *A = (double *)malloc(sizeof(double) * n * n);
    double *B = (double *)malloc(sizeof(double) * n * K);
    for (int r = 0; r < n; ++r)
        for (int cc = 0; cc < n; ++cc) A[r * n + cc] = ((r == cc) ? 1.0 : 0.0) - V[r * n + cc] * D[cc % M];
    for (int r = 0; r < n; ++r)
        for (int b = 0; b < K; ++b) B[r * K + b] = V[r * n + (b * M + NQ)];
    int rc = lu_solve(n, A, B, K);
    for (int a = 0; a < K; ++a)
        for (int b = 0; b < K; ++b) Kout[a * K + b] = B[(a * M + NQ) * K + b];
    free(xg); free(wg); free(k); free(w); free(D); free(V); free(A); free(B);
    return rc;
}

/* S from the on-shell K: T = (1 + i pi mu p K)^-1 K, S = 1 - 2 pi i mu p T. */
void or_S_from_K(int K, double p, const double *Km, double complex *S)
{
    double mu = or_mu();
    double complex x = I * OR_PI * mu * p;
    if (K == 1) {
        S[0] = (1.0 - x * Km[0]) / (1.0 + x * Km[0]);
        return;
    }
    double complex A[4] = {1.0 + x * Km[0], x * Km[1], x * Km[2], 1.0 + x * Km[3]};
    double complex Bm[4] = {1.0 - x * Km[0], -x * Km[1], -x * Km[2], 1.0 - x * Km[3]};
    double complex det = A[0] * A[3] - A[1] * A[2];
    double complex Ai[4] = {A[3] / det, -A[1] / det, -A[2] / det, A[0] / det};
    S[0] = Ai[0] * Bm[0] + Ai[1] * Bm[2];
    S[1] = Ai[0] * Bm[1] + Ai[1] * Bm[3];
    S[2] = Ai[2] * Bm[0] + Ai[3] * Bm[2];
    S[3] = Ai[2] * Bm[1] + Ai[3] * Bm[3];
}

static int batch_point(int n_ch, const int *chdesc, const int *nwp, const long *kb_off, const double *kb_all,
                       int wp_kind, int n_terms, const long *vt_off, const double *Vt_all, int n_samples,
                       const double *coeffs, int n_E, const double *e_lab, double complex *t_out, double *delta_out,
                       double *sigma_out, int n_threads)
{
    int err = 0;
    double *p = (double *)malloc(sizeof(double) * n_E);
    for (int e = 0; e < n_E; ++e) p[e] = or_p_of_tlab(e_lab[e]);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic) collapse(2)
#endif
    for (int smp = 0; smp < n_samples; ++smp)
        for (int c = 0; c < n_ch; ++c) {
            int K = chdesc[c * 6 + 4] ? 2 : 1;
            double complex *Tc = (double complex *)malloc(sizeof(double complex) * n_E * K * K);
            double *ph = (double *)malloc(sizeof(double) * n_E * 3);
            int rc = or_channel_solve_point(nwp[c], kb_all + kb_off[c], wp_kind, K, n_terms, Vt_all + vt_off[c],
                                            coeffs + (size_t)smp * (n_terms - 1), n_E, p, Tc, ph);
            if (rc < 0) {
#ifdef _OPENMP
#pragma omp critical(or_err)
#endif
                if (!err) err = rc;
            }
            for (int e = 0; e < n_E; ++e) {
                double complex *tout = t_out + (((size_t)smp * n_ch + c) * n_E + e) * 4;
                double *dout = delta_out + (((size_t)smp * n_ch + c) * n_E + e) * 3;
                for (int ab = 0; ab < 4; ++ab) tout[ab] = 0.0;
                for (int k = 0; k < 3; ++k) dout[k] = rc < 0 ? 0.0 : ph[3 * e + k];
                if (rc >= 0)
                    for (int a = 0; a < K; ++a)
                        for (int b = 0; b < K; ++b) tout[a * 2 + b] = Tc[(size_t)e * K * K + a * K + b];
            }
            free(Tc);
            free(ph);
        }
    for (int smp = 0; smp < n_samples; ++smp)
        for (int e = 0; e < n_E; ++e) {
            double acc = 0.0;
            for (int c = 0; c < n_ch; ++c)
                if (chdesc[c * 6 + 5] == 0)
                    acc += or_sigma_term(chdesc[c * 6 + 1], chdesc[c * 6 + 4] ? 2 : 1,
                                         delta_out + (((size_t)smp * n_ch + c) * n_E + e) * 3);
            sigma_out[(size_t)smp * n_E + e] = or_sigma_prefactor_mb(p[e]) * acc;
        }
    free(p);
    return err;
}

/* ------------------------------------------------------------------------- */
/* Batch driver used for the CPU baseline and the large parity cases: every   */
/* (sample, channel) is one channel-solve; the channel loop of each sample is */
/* followed by the interpolation and the cross-section sum.  Vt of channel c  */
/* starts at Vt_all + vt_off[c]; meshes per channel (kb_all + kb_off[c],     */
/* N = nwp[c]).  Outputs: t_out [S][n_ch][n_E][2][2] complex (continuum T of  */
/* the bin holding p(E)), delta_out [S][n_ch][n_E][3] deg, sigma_out [S][n_E] */
/* mb.  mode: 0 free-bin average, 1 SWP-bin average, 2 point resolvent (T    */
/* and phases at each p(E) directly).  OpenMP over (sample, channel).         */
/* Returns 0 or the first error code.                                         */
/* ------------------------------------------------------------------------- */
int or_batch_ip(int n_ch, const int *chdesc, const int *nwp, const long *kb_off, const double *kb_all, int wp_kind,
                int n_terms, const long *vt_off, const double *Vt_all, int n_samples, const double *coeffs, int n_E,
                const double *e_lab, int mode, double frac, double complex *t_out, double *delta_out,
                double *sigma_out, int n_threads);

int or_batch(int n_ch, const int *chdesc /* n_ch x 6 */, const int *nwp, const long *kb_off, const double *kb_all,
             int wp_kind, int n_terms, const long *vt_off, const double *Vt_all, int n_samples,
             const double *coeffs, int n_E, const double *e_lab, int mode, double complex *t_out, double *delta_out,
             double *sigma_out, int n_threads)
{
    return or_batch_ip(n_ch, chdesc, nwp, kb_off, kb_all, wp_kind, n_terms, vt_off, Vt_all, n_samples, coeffs, n_E,
                       e_lab, mode, 0.5, t_out, delta_out, sigma_out, n_threads);
}

/* or_batch with the interpolation point at fraction frac of each bin (Sec.  */
/* 5.1.1, Eq. "interpolation point"; 0 < frac < 1, 0.5 = the midpoints).     */
int or_batch_ip(int n_ch, const int *chdesc, const int *nwp, const long *kb_off, const double *kb_all, int wp_kind,
                int n_terms, const long *vt_off, const double *Vt_all, int n_samples, const double *coeffs, int n_E,
                const double *e_lab, int mode, double frac, double complex *t_out, double *delta_out,
                double *sigma_out, int n_threads)
{
    if (mode == 2) /* point resolvent: T and phases at each energy, no interpolation */
        return batch_point(n_ch, chdesc, nwp, kb_off, kb_all, wp_kind, n_terms, vt_off, Vt_all, n_samples, coeffs,
                           n_E, e_lab, t_out, delta_out, sigma_out, n_threads);
    int err = 0;
    long maxN = 0;
    for (int c = 0; c < n_ch; ++c)
        if (nwp[c] > maxN) maxN = nwp[c];
    double *phall = (double *)malloc(sizeof(double) * (size_t)n_samples * n_ch * maxN * 3);
    double complex *Tall = (double complex *)malloc(sizeof(double complex) * (size_t)n_samples * n_ch * maxN * 4);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic) collapse(2)
#endif
    for (int smp = 0; smp < n_samples; ++smp)
        for (int c = 0; c < n_ch; ++c) {
            int K = chdesc[c * 6 + 4] ? 2 : 1;
            int N = nwp[c], n = K * N;
            double *eps = (double *)malloc(sizeof(double) * n);
            double complex *Tc = Tall + ((size_t)smp * n_ch + c) * maxN * 4;
            double *ph = phall + ((size_t)smp * n_ch + c) * maxN * 3;
            int rc = or_channel_solve_ip(N, kb_all + kb_off[c], wp_kind, K, n_terms, Vt_all + vt_off[c],
                                         coeffs + (size_t)smp * (n_terms - 1), mode, frac, Tc, ph, eps, NULL);
            if (rc < 0) {
#ifdef _OPENMP
#pragma omp critical(or_err)
#endif
                if (!err) err = rc;
            }
            free(eps);
        }
    for (int smp = 0; smp < n_samples; ++smp)
        for (int e = 0; e < n_E; ++e) {
            double p = or_p_of_tlab(e_lab[e]);
            double acc = 0.0;
            for (int c = 0; c < n_ch; ++c) {
                int K = chdesc[c * 6 + 4] ? 2 : 1;
                int N = nwp[c];
                const double *kb = kb_all + kb_off[c];
                const double *ph = phall + ((size_t)smp * n_ch + c) * maxN * 3;
                const double complex *Tc = Tall + ((size_t)smp * n_ch + c) * maxN * 4;
                int bin = -1;
                for (int i = 0; i < N; ++i)
                    if (kb[i] <= p && p < kb[i + 1]) bin = i;
                double *dout = delta_out + (((size_t)smp * n_ch + c) * n_E + e) * 3;
                double complex *tout = t_out + (((size_t)smp * n_ch + c) * n_E + e) * 4;
                for (int ab = 0; ab < 4; ++ab) tout[ab] = 0.0;
                if (bin < 0) {
                    if (!err) err = -3;
                    dout[0] = dout[1] = dout[2] = 0.0;
                    continue;
                }
                for (int a = 0; a < K; ++a)
                    for (int b = 0; b < K; ++b) tout[a * 2 + b] = Tc[(size_t)bin * K * K + a * K + b];
                or_interp_phase_ip(N, kb, ph, K, p, frac, dout);
                if (chdesc[c * 6 + 5] == 0) acc += or_sigma_term(chdesc[c * 6 + 1], K, dout);
            }
            sigma_out[(size_t)smp * n_E + e] = or_sigma_prefactor_mb(p) * acc;
        }
    free(phall);
    free(Tall);
    return err;
}

/* ------------------------------------------------------------------------- */
/* Sec. 6 (method performance): the MI method solves the LS equation at n_I   */
/* energies of a Chebyshev distribution and interpolates the phase shifts     */
/* linearly between them.  Reading: linear in T_lab on the segment of         */
/* consecutive interpolation energies around the requested energy, the end    */
/* segments extended; delta moved by multiples of 180 deg to within 90 deg of  */
/* the segment's first value before interpolating (as for the midpoints).    */
/* e_int [n_I] ascending MeV; ph [n_I][3] degrees.                            */
/* ------------------------------------------------------------------------- */
void or_interp_phase_tlab(int n_I, const double *e_int, const double *ph, int K, double e, double *out)
{
    int j = -1;
    for (int i = 0; i < n_I; ++i)
        if (e_int[i] <= e) j = i;
    if (j < 0) j = 0;
    if (j > n_I - 2) j = n_I - 2;
    double w = (e - e_int[j]) / (e_int[j + 1] - e_int[j]);
    int ncomp = (K == 2) ? 2 : 1;
    for (int c = 0; c < ncomp; ++c) {
        double d0 = ph[3 * j + c], d1 = ph[3 * (j + 1) + c];
        d1 += 180.0 * round((d0 - d1) / 180.0);
        out[c] = wrap90(d0 + w * (d1 - d0));
    }
    if (K == 2) {
        out[2] = ph[3 * j + 2] + w * (ph[3 * (j + 1) + 2] - ph[3 * j + 2]);
    } else {
        out[1] = 0.0;
        out[2] = 0.0;
    }
}

/* MI batch: for every (sample, channel) the on-shell K at each interpolation */
/* energy (or_mi_kmatrix), S and the phases there, then the phases and the np */
/* total cross section at the requested energies by the interpolation above.  */
/* k_out [S][n_ch][n_I][2][2] (may be NULL), delta_out [S][n_ch][n_E][3],     */
/* sigma_out [S][n_E].  OpenMP over (sample, channel).  Returns 0 or the      */
/* first error code.                                                          */
int or_mi_batch(int n_ch, const int *chdesc, int gen, const double *gp, int n_terms, int n_samples,
                const double *coeffs, int NQ, double cmap, int n_I, const double *e_int, int n_E,
                const double *e_lab, double *k_out, double *delta_out, double *sigma_out, int n_threads)
{
    int err = 0;
    double *ph_all = (double *)malloc(sizeof(double) * (size_t)n_samples * n_ch * n_I * 3);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic) collapse(2)
#endif
    for (int smp = 0; smp < n_samples; ++smp)
        for (int c = 0; c < n_ch; ++c) {
            const int *d = chdesc + 6 * c;
            int K = d[4] ? 2 : 1;
            for (int e = 0; e < n_I; ++e) {
                double p = or_p_of_tlab(e_int[e]), Km[4];
                double complex S[4];
                int rc = or_mi_kmatrix(gen, gp, d[0], d[1], d[2], d[3], d[4], d[5], n_terms,
                                       coeffs + (size_t)smp * (n_terms - 1), NQ, cmap, p, Km);
                if (rc != 0) {
#ifdef _OPENMP
#pragma omp critical(or_err)
#endif
                    if (!err) err = -5;
                }
                if (k_out) {
                    double *ko = k_out + (((size_t)smp * n_ch + c) * n_I + e) * 4;
                    for (int ab = 0; ab < 4; ++ab) ko[ab] = 0.0;
                    for (int a = 0; a < K; ++a)
                        for (int b = 0; b < K; ++b) ko[a * 2 + b] = Km[a * K + b];
                }
                or_S_from_K(K, p, Km, S);
                or_phases_from_S(K, S, ph_all + (((size_t)smp * n_ch + c) * n_I + e) * 3);
            }
        }
    for (int smp = 0; smp < n_samples; ++smp)
        for (int e = 0; e < n_E; ++e) {
            double acc = 0.0;
            for (int c = 0; c < n_ch; ++c) {
                int K = chdesc[6 * c + 4] ? 2 : 1;
                double *dout = delta_out + (((size_t)smp * n_ch + c) * n_E + e) * 3;
                or_interp_phase_tlab(n_I, e_int, ph_all + ((size_t)smp * n_ch + c) * n_I * 3, K, e_lab[e], dout);
                if (chdesc[6 * c + 5] == 0) acc += or_sigma_term(chdesc[6 * c + 1], K, dout);
            }
            sigma_out[(size_t)smp * n_E + e] = or_sigma_prefactor_mb(or_p_of_tlab(e_lab[e])) * acc;
        }
    free(ph_all);
    return err;
}

/* ------------------------------------------------------------------------- */
/* App. A: spin observables of np scattering.  The M-matrix of Eq. "M-matrix */
/* PWE" with the incoming momentum along z, phi = 0 and momentum-space        */
/* partial waves (no i^(l-l') phase, consistent with the real symmetric K of  */
/* Sec. 2.1 and the Stapp S with its factor i in S_12), every np channel once */
/* (reading: the printed factor [1 - (-1)^(l+s+T_Z)] belongs to identical     */
/* nucleons; for np it would drop 1S0 and 3S1):                               */
/*   M^s_{m'm} = sqrt(4 pi)/(2 i p) sum_{J,l,l'} sqrt(2l+1)                   */
/*               C(l' (m-m') s m' | J m) C(l 0 s m | J m) (S_{l'l} - d_{l'l}) */
/*               Y_{l'}^{m-m'}(theta, 0).                                     */
/* The Saclay amplitudes a..e are the coefficients of M in the operator basis */
/* of Eq. "M matrix in terms of saclay amplitudes" (unit vectors l, m, n of   */
/* Eq. "kinematics vectors"), obtained by traces over the 4 x 4 two-nucleon    */
/* spin space; dsigma/dOmega = Tr(M M^dag)/4.  Reading: the e term is taken   */
/* along n, e (sigma_1 + sigma_2) . n -- the printed "m" would make it parity  */
/* odd (m is polar, n = p x p' axial), and only the n form completes the      */
/* basis of a parity-conserving M.                                            */
/* ------------------------------------------------------------------------- */
static double or_lfact(int n) { return lgamma((double)n + 1.0); }

/* Clebsch-Gordan <j1 m1 j2 m2 | J M> for integer spins (Racah's formula). */
double or_cg(int j1, int m1, int j2, int m2, int J, int M)
{
    if (m1 + m2 != M || abs(m1) > j1 || abs(m2) > j2 || abs(M) > J || J < abs(j1 - j2) || J > j1 + j2) return 0.0;
    double pre = 0.5 * (log(2.0 * J + 1.0) + or_lfact(J + j1 - j2) + or_lfact(J - j1 + j2) + or_lfact(j1 + j2 - J) -
                        or_lfact(j1 + j2 + J + 1) + or_lfact(J + M) + or_lfact(J - M) + or_lfact(j1 - m1) +
                        or_lfact(j1 + m1) + or_lfact(j2 - m2) + or_lfact(j2 + m2));
    double sum = 0.0;
    for (int k = 0; k <= j1 + j2 - J; ++k) {
        int a = j1 + j2 - J - k, b = j1 - m1 - k, c = j2 + m2 - k, d = J - j2 + m1 + k, e = J - j1 - m2 + k;
        if (a < 0 || b < 0 || c < 0 || d < 0 || e < 0) continue;
        double t = exp(pre - or_lfact(k) - or_lfact(a) - or_lfact(b) - or_lfact(c) - or_lfact(d) - or_lfact(e));
        sum += (k & 1) ? -t : t;
    }
    return sum;
}

/* Y_l^m(theta, phi = 0) with the Condon-Shortley phase. */
double or_ylm(int l, int m, double theta)
{
    int am = abs(m);
    if (am > l) return 0.0;
    double x = cos(theta), s = sin(theta);
    /* P_l^am without the Condon-Shortley phase by the upward recurrences */
    double pmm = 1.0;
    for (int i = 1; i <= am; ++i) pmm *= (2.0 * i - 1.0) * s;
    double plm = pmm;
    if (l > am) {
        double pm1 = x * (2.0 * am + 1.0) * pmm, pm0 = pmm;
        plm = pm1;
        for (int ll = am + 2; ll <= l; ++ll) {
            double pn = ((2.0 * ll - 1.0) * x * pm1 - (ll + am - 1.0) * pm0) / (ll - am);
            pm0 = pm1;
            pm1 = pn;
            plm = pn;
        }
    }
    double norm = sqrt((2.0 * l + 1.0) / (4.0 * OR_PI) * exp(or_lfact(l - am) - or_lfact(l + am)));
    double y = norm * plm * ((am & 1) ? -1.0 : 1.0); /* (-1)^m for m >= 0 */
    if (m < 0 && (am & 1)) y = -y;                    /* Y_l^{-m} = (-1)^m Y_l^m at phi = 0 */
    return y;
}

/* Partial-wave S of one channel from its (Stapp) phases, K x K. */
static void or_S_of_phases(int K, const double *phdeg, double complex *S)
{
    const double r = OR_PI / 180.0;
    if (K == 1) {
        S[0] = cexp(2.0 * I * phdeg[0] * r);
        return;
    }
    double dm = phdeg[0] * r, dp = phdeg[1] * r, e2 = 2.0 * phdeg[2] * r;
    S[0] = cos(e2) * cexp(2.0 * I * dm);
    S[3] = cos(e2) * cexp(2.0 * I * dp);
    S[1] = S[2] = I * sin(e2) * cexp(I * (dm + dp));
}

static void pauli_dot(const double *v, double complex out[2][2])
{
    out[0][0] = v[2];
    out[0][1] = v[0] - I * v[1];
    out[1][0] = v[0] + I * v[1];
    out[1][1] = -v[2];
}

static void kron2(double complex a[2][2], double complex b[2][2], double complex out[4][4])
{
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            for (int k = 0; k < 2; ++k)
                for (int l = 0; l < 2; ++l) out[2 * i + k][2 * j + l] = a[i][j] * b[k][l];
}

static double complex trace_prod(double complex A[4][4], double complex B[4][4])
{
    double complex t = 0.0;
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 4; ++k) t += A[i][k] * B[k][i];
    return t;
}

/* For every angle: the Saclay amplitudes abcde[t][5] (fm) and dsig[t]       */
/* (mb/sr) at momentum p from the phases ph [n_ch][3] (degrees) of the np     */
/* channels (tz = 0; others are skipped).  Also returns the M-matrix if       */
/* M_out is given: [t][4][4] in the product basis (up-up, up-down, down-up,   */
/* down-down).                                                                */
void or_saclay(int n_ch, const int *chdesc, const double *ph, double p, int n_th, const double *theta,
               double complex *abcde, double *dsig, double complex *M_out)
{
    for (int t = 0; t < n_th; ++t) {
        const double th = theta[t];
        double complex M0 = 0.0, M1[3][3]; /* M1[m'+1][m+1] */
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) M1[a][b] = 0.0;
        for (int c = 0; c < n_ch; ++c) {
            const int *d = chdesc + 6 * c;
            if (d[5] != 0) continue;
            int s = d[0], J = d[1], K = d[4] ? 2 : 1;
            int ls[2];
            ls[0] = d[4] ? J - 1 : d[2];
            ls[1] = d[4] ? J + 1 : d[2];
            double complex S[4];
            or_S_of_phases(K, ph + 3 * c, S);
            for (int ip = 0; ip < K; ++ip)
                for (int il = 0; il < K; ++il) {
                    int lp = ls[ip], l = ls[il];
                    double complex amp = S[ip * K + il] - (ip == il ? 1.0 : 0.0);
                    for (int m = -s; m <= s; ++m)
                        for (int mp = -s; mp <= s; ++mp) {
                            double w = sqrt(4.0 * OR_PI) * sqrt(2.0 * l + 1.0) * or_cg(lp, m - mp, s, mp, J, m) *
                                       or_cg(l, 0, s, m, J, m) * or_ylm(lp, m - mp, th);
                            if (w == 0.0) continue;
                            double complex v = w * amp / (2.0 * I * p);
                            if (s == 0) M0 += v;
                            else M1[mp + 1][m + 1] += v;
                        }
                }
        }
        /* to the product basis: |1,1> = uu, |1,0> = (ud+du)/sqrt2, |1,-1> = dd, |0,0> = (ud-du)/sqrt2 */
        double complex U[4][4] = {{0}}; /* columns: coupled states (1,1),(1,0),(1,-1),(0,0) */
        const double h = 1.0 / sqrt(2.0);
        U[0][0] = 1.0;
        U[1][1] = h;
        U[2][1] = h;
        U[3][2] = 1.0;
        U[1][3] = h;
        U[2][3] = -h;
        double complex Mc[4][4] = {{0}}, M[4][4];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Mc[2 - a][2 - b] = M1[a][b]; /* coupled index 0 <-> m = +1 */
        Mc[3][3] = M0;
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                double complex acc = 0.0;
                for (int k = 0; k < 4; ++k)
                    for (int l = 0; l < 4; ++l) acc += U[i][k] * Mc[k][l] * conj(U[j][l]);
                M[i][j] = acc;
            }
        /* unit vectors: l along p + p', m along p - p', n along p x p' */
        double lv[3] = {sin(0.5 * th), 0.0, cos(0.5 * th)}, mv[3] = {-cos(0.5 * th), 0.0, sin(0.5 * th)},
               nv[3] = {0.0, 1.0, 0.0};
        double complex sl[2][2], sm[2][2], sn[2][2], id[2][2] = {{1, 0}, {0, 1}};
        pauli_dot(lv, sl);
        pauli_dot(mv, sm);
        pauli_dot(nv, sn);
        double complex NN[4][4], MM[4][4], LL[4][4], S1[4][4], S2[4][4];
        kron2(sn, sn, NN);
        kron2(sm, sm, MM);
        kron2(sl, sl, LL);
        kron2(sn, id, S1); /* (sigma_1 + sigma_2) . n: the parity-even spin-orbit form (reading) */
        kron2(id, sn, S2);
        double complex trM = 0.0;
        for (int i = 0; i < 4; ++i) trM += M[i][i];
        double complex apb = 0.5 * trM, amb = 0.5 * trace_prod(M, NN), cpd = 0.5 * trace_prod(M, MM),
                       cmd = 0.5 * trace_prod(M, LL), e = 0.25 * (trace_prod(M, S1) + trace_prod(M, S2));
        double complex *o = abcde + (size_t)t * 5;
        o[0] = 0.5 * (apb + amb);
        o[1] = 0.5 * (apb - amb);
        o[2] = 0.5 * (cpd + cmd);
        o[3] = 0.5 * (cpd - cmd);
        o[4] = e;
        double tr = 0.0;
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) tr += creal(M[i][j] * conj(M[i][j]));
        dsig[t] = 0.25 * tr * 10.0; /* fm^2 -> mb */
        if (M_out)
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) M_out[(size_t)t * 16 + i * 4 + j] = M[i][j];
    }
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
