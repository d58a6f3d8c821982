// noalloc.cu -- one entry point that runs the per-channel hot path without
// allocating device memory.
//
// Some callers cannot call cudaMalloc: an application that owns all device
// memory through its own pool and forbids libraries from allocating, or a
// latency-critical loop that cannot take cudaMalloc's implicit device
// synchronisation.  For them wpcd_channel_solve_noalloc keeps every
// intermediate (mesh, eigenpairs, energy plan, bin-level T and phases) in one
// file-scope device array of fixed size, kScratchBytes, which every GPU that
// loads the library holds until the process exits.  The caller still passes
// its inputs and outputs.
//
// The array is shared by every call: calls whose work overlaps on the GPU
// (different streams, or different host threads) race on it.  Its device
// address is looked up once per device and kept: after cudaDeviceReset (or
// anything else that tears down and recreates the device's primary context)
// the module is loaded again and the array may move, so a process that resets
// a device must not call this entry point on it afterwards.  A call leaves
// its intermediates behind; each call rewrites everything it later reads, so
// nothing needs clearing between calls.
#include <mutex>

#include "wpcd_internal.cuh"

namespace wpcd {

constexpr size_t kScratchBytes = 16u << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

namespace {

// Device address of g_scratch per device: in host code the symbol's name is
// a host-side stand-in, so the address is looked up once per device with that
// device current.
std::mutex g_mu;
void *g_addr[64] = {};

cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

__global__ void k_store_chan(ChanDev cd, ChanDev *dst, int *list)
{
    *dst = cd;
    *list = 0;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace
}  // namespace wpcd

using namespace wpcd;

extern "C" wpcd_status wpcd_channel_solve_noalloc(int n_wp, int mesh_kind, double alpha_fm, double t, double kmax_fm,
                                                   int n_quad, int wp_kind, wpcd_channel ch, const double *V_dev,
                                                   int n_terms, const double *coeffs_dev, int n_samples,
                                                   const double *e_lab_dev, int n_E, double *t_out_dev,
                                                   double *delta_dev, int *status_dev, void *cuda_stream)
{
    if (n_wp < 4 || n_wp > kMaxNwp || n_quad < 1 || n_quad > kMaxQ || !(alpha_fm > 0) || !(t > 0) ||
        (mesh_kind != 0 && mesh_kind != 1) || (mesh_kind == 0 && !(kmax_fm > 0)) || (wp_kind != 0 && wp_kind != 1) ||
        !V_dev || n_terms < 1 || n_terms > kMaxTerms || (n_terms > 1 && !coeffs_dev) || n_samples < 1 ||
        !e_lab_dev || n_E < 1 || (!t_out_dev && !delta_dev))
        return WPCD_ERR_ARG;
    if (ch.coupled && (ch.s != 1 || ch.J < 1 || ch.l != ch.J - 1 || ch.lp != ch.J + 1)) return WPCD_ERR_ARG;
    if (!ch.coupled && ch.l != ch.lp) return WPCD_ERR_ARG;
    const int K = ch.coupled ? 2 : 1, N = n_wp, n = K * N, Q = n_quad;
    // matrices above one CTA's shared memory take the global-memory Jacobi
    // kernel with one scratch slot (its matrix and eigenvector copies) here
    const bool big = !jacobi_fits_smem(n, true);
    if (big && n > jacobi_big_max_n()) return WPCD_ERR_ARG;

    // carve the scratch array (every piece 256-byte aligned)
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return o;
    };
    const size_t o_chan = take(sizeof(ChanDev));
    const size_t o_glx = take(sizeof(double) * Q), o_glw = take(sizeof(double) * Q);
    const size_t o_kb = take(sizeof(double) * (N + 1)), o_kq = take(sizeof(double) * N * Q);
    const size_t o_wq = take(sizeof(double) * N * Q), o_h0 = take(sizeof(double) * N);
    const size_t o_list = take(sizeof(int));
    const size_t o_eps = take(sizeof(double) * (size_t)n_samples * n);
    const size_t o_C = take(sizeof(double) * (size_t)n_samples * n * n);
    const size_t o_status = take(sizeof(int) * (size_t)n_samples);
    const size_t o_bin = take(sizeof(int) * (size_t)n_E), o_brk = take(sizeof(int) * (size_t)n_E);
    const size_t o_cnt = take(sizeof(int)), o_plist = take(sizeof(int) * N), o_pE = take(sizeof(double) * n_E);
    const size_t o_tbin = take(sizeof(double) * (size_t)n_samples * N * 8);
    const size_t o_phbin = take(sizeof(double) * (size_t)n_samples * N * 3);
    const size_t o_big = big ? take(jacobi_big_scratch_bytes(n, true)) : 0;
    if (off > kScratchBytes) return WPCD_ERR_ARG;  // problem larger than the fixed scratch array

    void *base_v = nullptr;
    if (scratch_address(&base_v) != cudaSuccess) return WPCD_ERR_CUDA;
    unsigned char *base = static_cast<unsigned char *>(base_v);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    double *glx = reinterpret_cast<double *>(base + o_glx), *glw = reinterpret_cast<double *>(base + o_glw);
    double *kb = reinterpret_cast<double *>(base + o_kb), *kq = reinterpret_cast<double *>(base + o_kq);
    double *wq = reinterpret_cast<double *>(base + o_wq), *h0 = reinterpret_cast<double *>(base + o_h0);
    ChanDev *chan = reinterpret_cast<ChanDev *>(base + o_chan);
    int *list = reinterpret_cast<int *>(base + o_list);

    ChanDev cd{};
    cd.s = ch.s;
    cd.J = ch.J;
    cd.l = ch.l;
    cd.lp = ch.lp;
    cd.coupled = ch.coupled ? 1 : 0;
    cd.tz = ch.tz;
    cd.N = N;
    cd.K = K;
    cd.n = n;
    cd.Q = Q;
    cd.wp_kind = wp_kind;
    cd.kb = kb;
    cd.kq = kq;
    cd.wq = wq;
    cd.h0 = h0;
    cd.V = V_dev;
    cd.eps_off = 0;
    cd.c_off = 0;

    PlanDev plan{};  // one plan shared by all samples
    plan.bin = reinterpret_cast<int *>(base + o_bin);
    plan.brk = reinterpret_cast<int *>(base + o_brk);
    plan.cnt = reinterpret_cast<int *>(base + o_cnt);
    plan.list = reinterpret_cast<int *>(base + o_plist);
    plan.pE = reinterpret_cast<double *>(base + o_pE);
    double *eps = reinterpret_cast<double *>(base + o_eps), *C = reinterpret_cast<double *>(base + o_C);
    int *status = reinterpret_cast<int *>(base + o_status);
    double *tbin = reinterpret_cast<double *>(base + o_tbin), *phbin = reinterpret_cast<double *>(base + o_phbin);
    const double *cf = n_terms > 1 ? coeffs_dev : nullptr;

#define CKN(call)                                                  \
    do {                                                           \
        if ((call) != cudaSuccess) return WPCD_ERR_CUDA;           \
    } while (0)
    k_store_chan<<<1, 1, 0, counted(st)>>>(cd, chan, list);
    CKN(cudaGetLastError());
    CKN(launch_gauss_legendre(Q, glx, glw, st));
    CKN(launch_mesh(N, mesh_kind, alpha_fm, t, kmax_fm, Q, wp_kind, glx, glw, kb, kq, wq, h0, st));
    if (big)
        CKN(launch_jacobi_big(true, chan, list, 1, n_samples, 0, n_terms, cf, n, base + o_big, 1, eps, C, nullptr,
                              nullptr, nullptr, status, 1, status_dev, st));
    else
        CKN(launch_jacobi_f64(chan, list, 1, n_samples, 0, n_terms, cf, n, eps, C, status, 1, status_dev, st));
    CKN(launch_plan(chan, 1, N, e_lab_dev, n_E, plan, status_dev, st));
    CKN(launch_tbin(chan, 1, n_samples, n_terms, cf, eps, C, plan, N, n_E, tbin, phbin, status_dev, st, false,
                    WPCD_AVG_FREE_BIN));
    if (t_out_dev) CKN(launch_gather_t(chan, 1, n_samples, n_E, N, plan, tbin, t_out_dev, st));
    if (delta_dev) CKN(launch_observables(chan, 1, n_samples, n_E, N, plan, phbin, delta_dev, nullptr, st));
#undef CKN
    return WPCD_OK;
}
