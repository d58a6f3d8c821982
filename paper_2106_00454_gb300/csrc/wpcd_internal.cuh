// wpcd_internal.cuh -- types, constants and launch helpers shared by the
// CUDA translation units of libwpcd (sm_103a).  Not part of the C ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/wpcd.h"

namespace wpcd {

// Kinematics (the paper leaves the T_lab <-> p relation open): nonrelativistic
// p^2 = m_N T_lab / 2 with the np reduced-mass nucleon mass.
constexpr double kHbarc = 197.3269804;                // MeV fm
constexpr double kMn = 938.918309;                    // MeV, 2 m_p m_n/(m_p+m_n)
constexpr double kMu = 0.5 * kMn / kHbarc;            // reduced mass, fm^-1
constexpr double kPi = 3.14159265358979323846;

constexpr int kMaxNwp = 512;     // largest N_WP per channel
constexpr int kMaxQ = 16;        // largest fine points per bin
constexpr int kAngleQ = 96;      // Gauss-Legendre points in the scattering angle
constexpr int kMaxTerms = 16;    // potential terms per channel (V0 + 15)
constexpr int kYukTerms = 14;    // unit terms of the Yukawa/contact generator
constexpr int kYukParams = 19;
constexpr int kMaxJ = 16;

// Device error codes recorded in the context status word (first one wins).
enum DevErr : int {
    kDevOk = 0,
    kDevEnergyOutside = 1,
    kDevNoConverge = 2,
    kDevBranch = 3,
    kDevBadSize = 4,
    kDevMode = 5,    // resolvent mode not defined for this solve (SWP-bin average with a bound state)
    kDevTimeout = 6  // a bounded wait inside a kernel ran out
};

// Kernels launched by the calling host thread.  Every launch site passes its
// stream through counted(), so the runtime counts kernels exactly (including
// the ones a CUDA-graph capture records).
extern thread_local unsigned long long g_thread_kernels;
inline cudaStream_t counted(cudaStream_t st)
{
    ++g_thread_kernels;
    return st;
}

// Raise, never lower, a kernel's dynamic shared-memory limit to `bytes`.  The
// limit is a property of the kernel, and a CUDA graph captured earlier may
// hold a launch of the same kernel with more shared memory than the current
// launch needs, so the limit only grows (thread-safe).
cudaError_t raise_smem_limit(const void *kernel, size_t bytes);

// One channel of a projected potential set, as the kernels see it.
// Channel of an MI set: its grid potential terms Vg [n_terms][n][n] start at
// vg_off, its on-shell columns Von [n_I][n_terms][K][K][N_Q+1] at von_off;
// n = K (N_Q + 1).
struct MiChanDev {
    int s, J, l, lp, coupled, tz, K, n;
    long long vg_off, von_off;
};

// Channel of the spin-observable kernel: spin, J, T_z, K, its l values and the
// coupling products sqrt(4 pi) sqrt(2l+1) C(l' (m-m') s m' | J m) C(l 0 s m | J m)
// at tab[((l' block * 2 + l block) * 3 + m' + 1) * 3 + m + 1].
struct SacChanDev {
    int s, J, tz, K;
    int l[2];
    double tab[36];
};

struct ChanDev {
    int s, J, l, lp, coupled, tz;
    int N;              // N_WP of its mesh
    int K;              // 1 or 2 l-blocks
    int n;              // K * N
    int Q;              // fine points per bin
    int wp_kind;        // 0 momentum, 1 energy packets
    int pad_;
    const double *kb;   // mesh boundaries [N+1]
    const double *kq;   // fine nodes [N*Q]
    const double *wq;   // fine weights [N*Q]
    const double *h0;   // <x_i|h0|x_i> [N]
    const double *V;    // projected terms [n_terms][n][n]
    const double *d0;   // NULL, or the diagonal term [n] that replaces H0 (the eigensolvers only)
    long long eps_off;  // offset of this channel's eigenvalue block [S][n] in an eig buffer
    long long c_off;    // offset of this channel's eigenvector block [S][n][n]
};

// Energy plan: for each plan p (one shared by all samples, or one per sample
// when every sample carries its own energy list) and channel c.  n_E below is
// the stride of an energy list (its largest length).
struct PlanDev {
    int *bin;           // [P][n_ch][n_E] free bin holding p(E)
    int *brk;           // [P][n_ch][n_E] lower index j of the midpoint segment used to interpolate
    int *cnt;           // [P][n_ch] number of distinct bins whose T is needed
    int *list;          // [P][n_ch][maxN] those bins, ascending
    double *pE;         // [P][n_E] c.m. momentum of each energy
    int per_sample;     // 0: P = 1, the plan of every sample; 1: P = n_samples
    const int *n_E_s;   // per-sample list lengths (per_sample only; NULL = all n_E)
    double ip_frac = 0.5;  // interpolation point of a bin, as a fraction of it (0.5: the midpoint)
};

// Sec. 5.1.1, Eq. "interpolation point": the point k_i + f (k_{i+1} - k_i) of
// bin i at which its T is converted to the continuum and its phase placed for
// the interpolation, as (1 - f) k_i + f k_{i+1}; f = 1/2 gives exactly the
// midpoint 0.5 (k_i + k_{i+1}) (halving is exact, with or without a fused
// multiply-add).
__host__ __device__ __forceinline__ double ip_point(const double *kb, int i, double f)
{
    return (1.0 - f) * kb[i] + f * kb[i + 1];
}

__device__ __forceinline__ int plan_of(const PlanDev &pl, int smp) { return pl.per_sample ? smp : 0; }
__device__ __forceinline__ int plan_nE(const PlanDev &pl, int ps, int n_E) { return pl.n_E_s ? pl.n_E_s[ps] : n_E; }

// Bytes of dynamic shared memory this launch was given.
__device__ __forceinline__ unsigned dyn_smem_bytes()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

// S = 1 - 2 pi i mu q T from the continuum T (complex K x K, re/im interleaved,
// row-major in a 2 x 2 frame) and the phases in degrees: uncoupled delta =
// arg(S)/2; coupled (Stapp) delta_-, delta_+ = arg(S_11), arg(S_22) / 2 and
// eps_J = asin(Re[-i S_12 e^{-i(delta_- + delta_+)}]) / 2.  po: {delta or
// delta_-, delta_+, eps_J}.
__device__ __forceinline__ void phases_of_T(int K, double q, const double *T, double *po)
{
    // S = 1 - 2 pi i mu q T
    const double g = 2.0 * kPi * kMu * q;
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

// Shared-memory layouts (doubles) of the kernels, used by kernel and launcher alike.
__host__ __device__ inline size_t tbin_smem_doubles(int n)  // n = K * N of the channel
{
    // eps n, branch members 2n, branch boundaries 2(n+1), lo/hi/inverse widths 3n, X(E, B) at the two
    // bin edges 2(n+4), V rows 2n, R 2n, the six sums 8 and their per-thread terms 6 x 256 (the T
    // kernel's CTA size), diagonal V entries 4, per needed bin (<= n) edges, 1/dE, factor and index 4.5n
    return (size_t)14 * n + 2 + 8 + 8 + 6 * 256 + 4 + (size_t)5 * n;
}

__device__ __forceinline__ void record_error(int *err, int code)
{
    if (err) atomicCAS(err, 0, code);
}

// GB300 issues FP64 at 2 operations per clock per SM; conversions between
// FP64 and FP32 go through the bit patterns with integer operations instead.
// f32_trunc: x truncated to 24 significant bits (relative error < 2^-23),
// zero below the FP32 normal range.
__device__ __forceinline__ float f32_trunc(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int fe = (int)((b >> 52) & 0x7FF) - 1023 + 127;
    if (fe <= 0) return 0.0f;
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    if (fe >= 255) return __uint_as_float(sign | 0x7F800000u);
    return __uint_as_float(sign | ((unsigned)fe << 23) | (unsigned)((b >> 29) & 0x7FFFFFu));
}

// The FP32 value as FP64 (exact; FP32 subnormals, below 1.2e-38, become zero).
__device__ __forceinline__ double f64_of(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned fe = (u >> 23) & 0xFF;
    if (fe == 0) return 0.0;
    const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                                 ((unsigned long long)(fe - 127 + 1023) << 52) |
                                 ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)b);
}

// Packed upper-triangle index (i <= j), column-major: element (i, j) at j(j+1)/2 + i.
__device__ __forceinline__ int pk(int i, int j)
{
    return (i <= j) ? (j * (j + 1) / 2 + i) : (i * (i + 1) / 2 + j);
}

// Round-robin tournament (npad even): pair k of round r.  Every unordered pair
// of 0..npad-1 occurs in exactly one of the npad-1 rounds; each round is a
// perfect matching, so its rotations commute.
__device__ __forceinline__ void jac_pair_of(int r, int k, int npad, int &p, int &q)
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

// Sum of one double over the CTA (blockDim a multiple of 32, <= 2048); every thread gets it.
__device__ __forceinline__ double cta_sum64(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

}  // namespace wpcd

// ---- host-side launch interfaces (defined in the .cu files) ----------------------------------
namespace wpcd {

cudaError_t launch_gauss_legendre(int n, double *x, double *w, cudaStream_t st);
cudaError_t launch_mesh(int N, int kind, double alpha, double t, double kmax, int Q, int wp_kind,
                        const double *glx, const double *glw, double *kb, double *kq, double *wq, double *h0,
                        cudaStream_t st);
cudaError_t launch_project_yukawa(const ChanDev *chans_dev, const int *group_dev, int n_group, int N, int Q,
                                  int Lmax, const double *gp_dev, const double *angx, const double *angw,
                                  int n_terms, cudaStream_t st, const float *Ibuf = nullptr);
size_t angle_tc_buffer_bytes(int N, int Q);
cudaError_t launch_angle_tc(const ChanDev *chans_dev, const int *group_dev, int N, int Q, int Lm, const double *gp_dev,
                            const double *angx, const double *angw, float *Iout, int *err, cudaStream_t st);
cudaError_t launch_project_yamaguchi_gp(const ChanDev *chans_dev, const int *group_dev, int n_group, int N, int Q,
                                        const double *gp_dev, cudaStream_t st);
cudaError_t launch_project_fine(const ChanDev *chans_dev, int c, const ChanDev &ch_host, const double *vfine,
                                int n_terms, cudaStream_t st);
size_t jacobi_smem_bytes(int n, bool c_in_smem);
bool jacobi_c_in_smem(int n);
cudaError_t launch_jacobi_f64(const ChanDev *chans_dev, const int *work_ch_dev, int n_work_ch, int n_samples,
                              int sample0, int n_terms, const double *coeffs, int n, double *eps_all,
                              double *C_all, int *status_all, int n_ch_total, int *err, cudaStream_t st,
                              int threads = 256);
int jacobi_f64_occupancy(int n, int threads);
int jacobi_mixed_occupancy(int n, int threads);
bool jacobi_mixed_c_in_smem(int n);   // eigenvector matrix in shared memory (else global)
size_t jacobi_mixed_smem_bytes(int n, bool c_in_smem);
size_t jacobi_mixed_c_bytes(int n);  // global eigenvector scratch per item (C kept in global memory)
cudaError_t launch_jacobi_mixed(const ChanDev *chans_dev, const int *work_ch_dev, int n_work_ch, int n_samples,
                                int sample0, int n_terms, const double *coeffs, int n, double *lam_s, double *X_s,
                                float *Cf_s, double *H_s, int *status_all, int n_ch_total, int *err, cudaStream_t st,
                                int threads = 256);
// Matrices above one CTA's shared memory: Jacobi with A and C in global memory.
bool jacobi_fits_smem(int n, bool f64);
int jacobi_big_max_n();
int jacobi_big_occupancy(int n, bool f64);
size_t jacobi_big_scratch_bytes(int n, bool f64);
cudaError_t launch_jacobi_big(bool f64, const ChanDev *chans_dev, const int *work_ch_dev, int n_work_ch,
                              int n_samples, int sample0, int n_terms, const double *coeffs, int n, void *scratch,
                              int slots, double *eps_all, double *C_all, double *lam_s, double *X_s, double *H_s,
                              int *status_all, int n_ch_total, int *err, cudaStream_t st);
constexpr int kOzDigits = 6;  // balanced 8-bit digits per operand of the Ozaki products
size_t oz_slice_elems(int n);
int oz_kpad(int n);
cudaError_t launch_oz_gemm(int n, int items, bool ta, const double *A, const double *B, double *C,
                           __nv_bfloat16 *sa, __nv_bfloat16 *sb, int *ea, int *eb, cudaStream_t st, int *err = nullptr);
cudaError_t launch_oz_split(int n, int items, bool cols, const double *M, __nv_bfloat16 *S, int *e, cudaStream_t st);
cudaError_t launch_oz_gemm_slices(int n, int items, const __nv_bfloat16 *sa, const int *ea, const __nv_bfloat16 *sb,
                                  const int *eb, double *C, cudaStream_t st, int digits = 6, bool sym = false,
                                  int *err = nullptr, int a_items = 0);
cudaError_t launch_oz_gemm_tc(int n, int items, const __nv_bfloat16 *sa, const int *ea, const __nv_bfloat16 *sb,
                              const int *eb, double *C, int digits, bool sym, int *err, cudaStream_t st,
                              int a_items = 0);
size_t refine_scratch_per_item(int n, int engine);
cudaError_t launch_refine(const ChanDev *chans, const int *work, int nw, int n_samples, int sample0, int n,
                          int n_terms, const double *coeffs, void *scratch, double *eps_all, double *X_all,
                          int iters, int engine, cudaStream_t st, int *err = nullptr,
                          const __nv_bfloat16 *rot_s = nullptr, const int *rot_e = nullptr, int digits = 6);
cudaError_t launch_batched_dgemm(int n, int items, bool ta, const double *A, const double *B, double *C,
                                 void *scratch, int engine, cudaStream_t st, int *err = nullptr);
size_t batched_dgemm_scratch(int n, int items);
cudaError_t launch_plan(const ChanDev *chans_dev, int n_ch, int maxN, const double *e_lab, int n_E, PlanDev plan,
                        int *err, cudaStream_t st, int n_plans = 1);
cudaError_t launch_tbin(const ChanDev *chans_dev, int n_ch, int n_samples, int n_terms, const double *coeffs,
                        const double *eps_all, const double *C_all, PlanDev plan, int maxN, int n_E, double *tout,
                        double *phout, int *err, cudaStream_t st, bool vc_identity, int mode);
cudaError_t launch_saclay(const SacChanDev *chans_dev, int n_ch, int n_samples, int n_E, const double *e_lab,
                          const double *delta, int n_th, const double *theta, double *abcde, double *dsig,
                          cudaStream_t st);
constexpr int kMiMaxNQ = 100;  // MI grid points per l-block: 2 (N_Q + 1) rows fit one CTA's shared memory in FP32
cudaError_t launch_mi_grid(int NQ, double cmap, const double *glx, const double *glw, double *k, double *w,
                           cudaStream_t st);
cudaError_t launch_mi_pot(int gen, const MiChanDev *chans_dev, int n_ch, int NQ, const double *kg, int Lmax,
                          const double *gp_dev, const double *angx, const double *angw, int n_terms, double *Vg,
                          cudaStream_t st);
cudaError_t launch_mi_onshell(int gen, const MiChanDev *chans_dev, int n_ch, int NQ, const double *kg, int n_I,
                              const double *e_int, int Lmax, const double *gp_dev, const double *angx,
                              const double *angw, int n_terms, double *Von, cudaStream_t st);
cudaError_t launch_mi_solve(const MiChanDev *chans_dev, const int *work_dev, int n_work, int n, int n_ch_total,
                            int n_samples, int NQ, const double *kg, const double *wg, int n_terms,
                            const double *coeffs, const double *Vg, const double *Von, int n_I, const double *e_int,
                            double *Vs, int slots, double *ph, double *k_out, int *status, int *err,
                            cudaStream_t st);
int mi_slots_per_sm(int n, int NQ);
cudaError_t launch_mi_observables(const MiChanDev *chans_dev, int n_ch, int n_samples, int n_I, const double *e_int,
                                  const double *ph, int n_E, const double *e_lab, double *delta, double *sigma,
                                  cudaStream_t st);
cudaError_t launch_wlog(const double *x, double *y, int n, cudaStream_t st);
cudaError_t launch_gather_t(const ChanDev *chans_dev, int n_ch, int n_samples, int n_E, int maxN, PlanDev plan,
                            const double *tbin, double *t_out, cudaStream_t st, bool direct = false);
cudaError_t launch_observables(const ChanDev *chans_dev, int n_ch, int n_samples, int n_E, int maxN, PlanDev plan,
                               const double *phbin, double *delta, double *sigma, cudaStream_t st,
                               bool direct = false);

}  // namespace wpcd
