// runtime.cu -- host runtime of libwpcd: context, handle tables, device-memory
// accounting against the HBM budget, size buckets, and the C ABI of wpcd.h.
// Every numerical step runs in the kernels of the other translation units;
// this file only allocates, validates, orders launches and copies.
#include <algorithm>
#include <array>
#include <cmath>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "wpcd_internal.cuh"

namespace wpcd {
size_t tbin_smem_bytes(int nmax);
thread_local unsigned long long g_thread_kernels = 0;

cudaError_t raise_smem_limit(const void *kernel, size_t bytes)
{
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    if (e != cudaSuccess || (size_t)a.maxDynamicSharedSizeBytes >= bytes) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
}

using namespace wpcd;

namespace {

constexpr size_t kRefineScratchBytes = (size_t)32 << 30;  // mixed path: refinement scratch per bucket chunk (one chunk per bucket up to ~7000 samples of n = 200)
constexpr int kRefineIters = 2;                            // FP64 refinement iterations (default)
constexpr size_t kGraphCache = 64;                         // wpcd_solve keys remembered for CUDA graphs

struct MeshH {
    int N = 0, Q = 0, kind = 0, wp_kind = 0;
    double alpha = 0, t = 0, kmax = 0;
    double *kb = nullptr, *kq = nullptr, *wq = nullptr, *h0 = nullptr;
};

struct VSetH {
    int n_ch = 0, n_terms = 0, gen = 0, maxN = 0, maxn = 0;
    std::vector<wpcd_channel> ch;
    std::vector<int> mesh_ids;
    std::vector<ChanDev> cd;  // host copy (V pointers filled, offsets zero)
    double *V = nullptr;
    ChanDev *cd_dev = nullptr;
    std::map<int, std::vector<int>> buckets;  // n -> channel indices
    std::map<int, int *> bucket_dev;          // n -> device list of channel indices
    int *ident_dev = nullptr;                 // [n_ch] = 0..n_ch-1 (plain mode)
    // Mean-potential eigenbasis of the mixed path (built on first use): per channel
    // C0, eps0 = eig(diag(H0) + V0) in FP64 and the rotated terms W_a = C0^T V_a C0
    // (W_0 = 0), so that C0^T H(c) C0 = diag(eps0) + sum_a c_a W_a; per size bucket
    // the digit slices of the rows of its channels' C0 for the back-rotation X = C0 X'.
    struct RotB {
        double *C0 = nullptr;  // [nw][n][n], the bucket's channels in bucket order
        __nv_bfloat16 *sC = nullptr;
        int *eC = nullptr;
    };
    std::unique_ptr<std::mutex> rot_mu{new std::mutex};
    int rot_state = 0;  // 0 not built, 1 ready, -1 failed (the mixed path then runs in the original basis)
    double *Vr = nullptr, *eps0 = nullptr, *C0 = nullptr;
    std::vector<ChanDev> cd_rot;  // host copy: V -> W_a, d0 -> eps0 (offsets zero)
    std::map<int, RotB> rotb;
};

struct EigH {
    int vset_id = -1, n_samples = 0, prec = WPCD_PREC_FP64;
    double *eps = nullptr, *C = nullptr, *coeffs = nullptr;
    // (the mixed path leaves refined FP64 eigenpairs in eps / C as well)
    int *status = nullptr;
    ChanDev *cd_dev = nullptr;      // vset channels with this eig's offsets
    ChanDev *cd_rot_dev = nullptr;  // the same in the mean-potential eigenbasis (mixed path)
    bool rot = false;               // this batch's eigensolve runs in that basis
    size_t eps_len = 0, c_len = 0, coeff_len = 0, status_len = 0, cd_len = 0;
};

// Grow-only device buffer.
struct Buf {
    void *p = nullptr;
    size_t n = 0;
};

// One executor: a stream, its device status word and its workspaces.  The
// synchronous API runs on the context's own executor; each serving slot has
// one of its own so that batches overlap on the device.
struct Exec {
    cudaStream_t stream = nullptr;
    int *err = nullptr;
    Buf ws_plan_i, ws_plan_d, ws_tbin, ws_phbin, ws_ref, ws_in, ws_out;
    EigH eig;
};

// MI set: the momentum grid, the channels and their grid potential terms.
struct MiH {
    int n_ch = 0, NQ = 0, n_terms = 0, gen = 0, Lmax = 0, n_gp = 0;
    double cmap = 1.0;
    std::vector<MiChanDev> ch;
    MiChanDev *ch_dev = nullptr;
    double *kg = nullptr, *wg = nullptr, *gp = nullptr, *Vg = nullptr;
    int *work_dev[2] = {nullptr, nullptr};  // channels with K = 1, 2
    int n_work[2] = {0, 0};
};

enum Kind { kMesh = 1, kVSet = 2, kEig = 3, kMi = 4 };

struct Handle {
    Kind kind;
    std::unique_ptr<MeshH> mesh;
    std::unique_ptr<VSetH> vset;
    std::unique_ptr<EigH> eig;
    std::unique_ptr<MiH> mi;
};

}  // namespace

struct wpcd_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t budget = 0, in_use = 0;
    std::map<void *, size_t> sizes;
    std::map<int, Handle> handles;
    int next_id = 1;
    std::mutex mu;
    int exec_mode = WPCD_EXEC_BATCHED;
    int refine_engine = WPCD_REFINE_TENSOR;
    int rotate = 1;  // mixed path in the mean-potential eigenbasis (WPCD_OPT_ROTATE)
    int refine_iters = kRefineIters;  // WPCD_OPT_REFINE_ITERS
    int refine_digits = 6;            // WPCD_OPT_REFINE_DIGITS
    int autotune = 1;
    int n_sm = 0;
    struct Tuned {
        int threads;
        float ms[5];
    };
    std::map<std::pair<int, int>, Tuned> tuned;  // (n, precision) -> eigensolver CTA size
    std::mutex tmu;
    int *err_dev = nullptr;
    std::mutex amu;  // device-memory accounting (shared with the serving thread)
    std::mutex pmu;  // profiling records
    // Gauss-Legendre rules cached on the device, keyed by order
    std::map<int, std::pair<double *, double *>> gl;
    Exec main;  // executor of the synchronous API (the caller's stream)
    struct Server *server = nullptr;
    // tracing: kernels launched, and (when enabled) CUDA events around each launch
    std::atomic<unsigned long long> launches{0};
    bool prof = false;
    struct Rec {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    double prof_ms[WPCD_PHASE_COUNT] = {};
    long prof_n[WPCD_PHASE_COUNT] = {};
    // CUDA graphs of wpcd_solve.  graph_gen counts every event that may change
    // what a captured graph baked in (a device allocation or free, an option, a
    // new tuning); a graph captured under another generation is dropped.
    double ip_frac = 0.5;  // interpolation point of the averaged resolvents (Sec. 5.1.1)
    int big_slots = 0;     // CTAs of the global-memory eigensolver (0: automatic)
    int use_graphs = 1;
    std::atomic<unsigned long long> graph_gen{0};
    struct GraphE {
        unsigned long long gen = 0;  // generation when first seen / captured
        cudaGraphExec_t exec = nullptr;
        unsigned long long kernels = 0;  // kernels the graph holds
        bool failed = false;             // capture failed: stay one by one
    };
    std::map<std::array<unsigned long long, 12>, GraphE> graphs;
    cudaStream_t cap_stream = nullptr;  // private stream the captures run on
    unsigned long long graph_captures = 0, graph_replays = 0;
};

namespace {

#define CK(call)                                      \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return WPCD_ERR_CUDA; \
    } while (0)

wpcd_status dmalloc(wpcd_ctx *c, void **p, size_t bytes)
{
    std::lock_guard<std::mutex> lk(c->amu);
    if (bytes == 0) bytes = 8;
    if (c->budget && c->in_use + bytes > c->budget) return WPCD_ERR_BUDGET;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return WPCD_ERR_NOMEM;
    }
    c->in_use += bytes;
    c->sizes[*p] = bytes;
    ++c->graph_gen;
    return WPCD_OK;
}

void dfree(wpcd_ctx *c, void *p)
{
    if (!p) return;
    std::lock_guard<std::mutex> lk(c->amu);
    auto it = c->sizes.find(p);
    if (it != c->sizes.end()) {
        c->in_use -= it->second;
        c->sizes.erase(it);
    }
    ++c->graph_gen;
    cudaFree(p);
}

template <class T>
wpcd_status dalloc(wpcd_ctx *c, T **p, size_t count)
{
    return dmalloc(c, reinterpret_cast<void **>(p), count * sizeof(T));
}

// One launch step of `phase` (one or more kernels): adds the kernels it
// launched to the context count; with profiling on, brackets it with events.
struct Launch {
    wpcd_ctx *c;
    cudaStream_t st;
    wpcd_ctx::Rec r{};
    bool on;
    unsigned long long k0;
    Launch(wpcd_ctx *cc, const Exec &X, int phase) : c(cc), st(X.stream), on(cc->prof), k0(g_thread_kernels)
    {
        r.phase = phase;
        if (on) {
            cudaEventCreate(&r.a);
            cudaEventCreate(&r.b);
            cudaEventRecord(r.a, st);
        }
    }
    ~Launch()
    {
        c->launches += g_thread_kernels - k0;
        if (on) {
            cudaEventRecord(r.b, st);
            std::lock_guard<std::mutex> lk(c->pmu);
            c->recs.push_back(r);
        }
    }
};

void prof_collect(wpcd_ctx *c)
{
    std::lock_guard<std::mutex> lk(c->pmu);
    if (c->recs.empty()) return;
    for (auto &r : c->recs) {
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        c->prof_ms[r.phase] += ms;
        c->prof_n[r.phase] += 1;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    c->recs.clear();
}

bool capturing(cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

wpcd_status ws_reserve(wpcd_ctx *c, const Exec &X, Buf &b, size_t bytes)
{
    if (b.n >= bytes) return WPCD_OK;
    if (capturing(X.stream)) return WPCD_ERR_CUDA;  // a graph cannot hold a reallocation
    if (b.p) {
        cudaStreamSynchronize(X.stream);
        dfree(c, b.p);
        b.p = nullptr;
        b.n = 0;
    }
    wpcd_status st = dmalloc(c, &b.p, bytes);
    if (st == WPCD_OK) b.n = bytes;
    return st;
}

wpcd_status gl_rule(wpcd_ctx *c, int n, double **x, double **w)
{
    auto it = c->gl.find(n);
    if (it != c->gl.end()) {
        *x = it->second.first;
        *w = it->second.second;
        return WPCD_OK;
    }
    double *dx, *dw;
    wpcd_status st = dalloc(c, &dx, n);
    if (st) return st;
    st = dalloc(c, &dw, n);
    if (st) {
        dfree(c, dx);
        return st;
    }
    {
        Launch L(c, c->main, WPCD_PHASE_MESH);
        CK(launch_gauss_legendre(n, dx, dw, c->main.stream));
    }
    c->gl[n] = {dx, dw};
    *x = dx;
    *w = dw;
    return WPCD_OK;
}

Handle *find(wpcd_ctx *c, int id, Kind k)
{
    auto it = c->handles.find(id);
    if (it == c->handles.end() || it->second.kind != k) return nullptr;
    return &it->second;
}

void free_eig(wpcd_ctx *c, EigH &e)
{
    dfree(c, e.eps);
    dfree(c, e.C);
    dfree(c, e.coeffs);
    dfree(c, e.status);
    dfree(c, e.cd_dev);
    dfree(c, e.cd_rot_dev);
    e = EigH();
}

void free_vset(wpcd_ctx *c, VSetH &v)
{
    dfree(c, v.V);
    dfree(c, v.cd_dev);
    dfree(c, v.ident_dev);
    for (auto &kv : v.bucket_dev) dfree(c, kv.second);
    dfree(c, v.Vr);
    dfree(c, v.eps0);
    dfree(c, v.C0);
    for (auto &kv : v.rotb) {
        dfree(c, kv.second.sC);
        dfree(c, kv.second.eC);
    }
}

void free_mi(wpcd_ctx *c, MiH &m)
{
    dfree(c, m.ch_dev);
    dfree(c, m.kg);
    dfree(c, m.wg);
    dfree(c, m.gp);
    dfree(c, m.Vg);
    dfree(c, m.work_dev[0]);
    dfree(c, m.work_dev[1]);
}

void free_mesh(wpcd_ctx *c, MeshH &m)
{
    dfree(c, m.kb);
    dfree(c, m.kq);
    dfree(c, m.wq);
    dfree(c, m.h0);
}

// Autotuner of the eigensolver's CTA size.  On the first batched use of a
// (matrix size, precision) it times each candidate on about two full waves of
// the bucket's own solves (occupancy from the CUDA occupancy calculator) and
// keeps the fastest; the tuning launches write the same outputs the real
// launch then overwrites.  Returns the CTA size, or -1 on a CUDA error.
template <class F>
int pick_threads(wpcd_ctx *c, Exec &X, int n, int prec, int nw, int nsmp, F launch)
{
    static const int cand[5] = {64, 128, 256, 512, 1024};  // 1024: the FP32 kernel only
    if (!c->autotune || c->exec_mode != WPCD_EXEC_BATCHED) return 256;
    const auto key = std::make_pair(n, prec);
    {
        std::lock_guard<std::mutex> lk(c->tmu);
        auto it = c->tuned.find(key);
        if (it != c->tuned.end()) return it->second.threads;
    }
    if (capturing(X.stream)) return -1;  // tuning synchronises: never inside a capture
    if (!c->n_sm) cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);
    wpcd_ctx::Tuned t{256, {-1.f, -1.f, -1.f, -1.f, -1.f}};
    float best = 1e30f;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    for (int k = 0; k < 5; ++k) {
        const int th = cand[k];
        if (th > 512 && prec == WPCD_PREC_FP64) continue;
        if (prec == WPCD_PREC_FP64 && !jacobi_c_in_smem(n) && (th / 32) * n > n * (n + 1) / 2) continue;
        const int occ = prec == WPCD_PREC_FP64 ? jacobi_f64_occupancy(n, th) : jacobi_mixed_occupancy(n, th);
        if (occ < 1) continue;
        const int ns = std::max(1, std::min(nsmp, (2 * c->n_sm * occ + nw - 1) / nw));
        cudaEventRecord(a, X.stream);
        if (launch(th, ns) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        cudaEventRecord(b, X.stream);
        if (cudaEventSynchronize(b) != cudaSuccess) {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            return -1;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        const float per = ms / (float)(ns * nw);  // time per solve
        t.ms[k] = per;
        if (per < best) {
            best = per;
            t.threads = th;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    std::lock_guard<std::mutex> lk(c->tmu);
    c->tuned[key] = t;
    ++c->graph_gen;
    return t.threads;
}

// Build the mean-potential eigenbasis of a vset (once, on the executor's
// stream, synchronising; concurrent callers wait on the vset's lock):
//   C0, eps0 = eig(diag(H0) + V0) with the FP64 Jacobi kernels;
//   W_a = C0^T V_a C0 (a >= 1) with FP64 products, W_0 = 0;
//   per size bucket, the digit slices of the rows of its channels' C0.
// The FP32 eigensolve of the mixed path then starts from C0^T H C0 =
// diag(eps0) + sum_a c_a W_a, an orthogonal similarity of H that is nearly
// diagonal for parameter samples near the mean (fewer Jacobi sweeps), and the
// refined eigenvectors are rotated back, X = C0 X'.
wpcd_status ensure_rotation(wpcd_ctx *c, Exec &X, VSetH &v)
{
    std::lock_guard<std::mutex> lk(*v.rot_mu);
    if (v.rot_state != 0) return WPCD_OK;
    v.rot_state = -1;
    size_t ne = 0, nc = 0, vlen = 0;
    int nmax = 0;
    std::vector<ChanDev> cd = v.cd;  // offsets of a one-sample eigen buffer, bucket by bucket
    std::map<int, size_t> bstart;
    for (auto &kv : v.buckets) {
        bstart[kv.first] = nc;
        for (int k : kv.second) {
            cd[k].eps_off = (long long)ne;
            cd[k].c_off = (long long)nc;
            ne += cd[k].n;
            nc += (size_t)cd[k].n * cd[k].n;
        }
    }
    for (auto &d : v.cd) {
        vlen += (size_t)v.n_terms * d.n * d.n;
        nmax = std::max(nmax, d.n);
    }
    wpcd_status st;
    if ((st = dalloc(c, &v.eps0, ne)) || (st = dalloc(c, &v.C0, nc)) || (st = dalloc(c, &v.Vr, vlen))) return st;
    ChanDev *cd_tmp = nullptr;
    int *status = nullptr;
    void *big = nullptr;
    double *Crep = nullptr, *T = nullptr;
    auto cleanup = [&]() {
        cudaStreamSynchronize(X.stream);
        dfree(c, cd_tmp);
        dfree(c, status);
        dfree(c, big);
        dfree(c, Crep);
        dfree(c, T);
    };
    if ((st = dalloc(c, &cd_tmp, (size_t)v.n_ch)) || (st = dalloc(c, &status, (size_t)v.n_ch))) {
        cleanup();
        return st;
    }
    CK(cudaMemcpyAsync(cd_tmp, cd.data(), sizeof(ChanDev) * v.n_ch, cudaMemcpyHostToDevice, X.stream));
    for (auto &kv : v.buckets) {
        const int n = kv.first, nw = (int)kv.second.size();
        if (jacobi_fits_smem(n, true)) {
            CK(launch_jacobi_f64(cd_tmp, v.bucket_dev[n], nw, 1, 0, 1, nullptr, n, v.eps0, v.C0, status, v.n_ch,
                                 X.err, X.stream, 256));
        } else {
            const size_t slot_b = (jacobi_big_scratch_bytes(n, true) + 255) & ~(size_t)255;
            cudaStreamSynchronize(X.stream);
            dfree(c, big);
            big = nullptr;
            if ((st = dmalloc(c, &big, slot_b * nw))) {
                cleanup();
                return st;
            }
            CK(launch_jacobi_big(true, cd_tmp, v.bucket_dev[n], nw, 1, 0, 1, nullptr, n, big, nw, v.eps0, v.C0,
                                 nullptr, nullptr, nullptr, status, v.n_ch, X.err, X.stream));
        }
    }
    const int na = v.n_terms - 1;
    if (na > 0 && ((st = dalloc(c, &Crep, (size_t)na * nmax * nmax)) || (st = dalloc(c, &T, (size_t)na * nmax * nmax)))) {
        cleanup();
        return st;
    }
    for (int k = 0; k < v.n_ch; ++k) {
        const int n = cd[k].n;
        const size_t nn = (size_t)n * n;
        double *Vr_k = v.Vr + (v.cd[k].V - v.V);
        CK(cudaMemsetAsync(Vr_k, 0, nn * sizeof(double), X.stream));  // W_0 = 0
        if (na == 0) continue;
        for (int a = 0; a < na; ++a)
            CK(cudaMemcpyAsync(Crep + (size_t)a * nn, v.C0 + cd[k].c_off, nn * sizeof(double),
                               cudaMemcpyDeviceToDevice, X.stream));
        CK(launch_batched_dgemm(n, na, false, v.cd[k].V + nn, Crep, T, nullptr, WPCD_REFINE_FP64, X.stream));
        CK(launch_batched_dgemm(n, na, true, Crep, T, Vr_k + nn, nullptr, WPCD_REFINE_FP64, X.stream));
    }
    for (auto &kv : v.buckets) {
        const int n = kv.first, nw = (int)kv.second.size();
        VSetH::RotB &rb = v.rotb[n];
        rb.C0 = v.C0 + bstart[n];
        if ((st = dalloc(c, &rb.sC, (size_t)nw * oz_slice_elems(n))) || (st = dalloc(c, &rb.eC, (size_t)nw * n))) {
            cleanup();
            return st;
        }
        CK(launch_oz_split(n, nw, false, rb.C0, rb.sC, rb.eC, X.stream));
    }
    std::vector<int> hs(v.n_ch);
    int herr = 0;
    CK(cudaMemcpyAsync(hs.data(), status, sizeof(int) * v.n_ch, cudaMemcpyDeviceToHost, X.stream));
    CK(cudaMemcpyAsync(&herr, X.err, sizeof(int), cudaMemcpyDeviceToHost, X.stream));
    cleanup();
    bool ok = herr == 0;
    for (int k = 0; k < v.n_ch; ++k) ok &= hs[k] >= 0;
    if (!ok) return WPCD_OK;  // stays -1: the mixed path keeps the original basis
    v.cd_rot = v.cd;
    for (int k = 0; k < v.n_ch; ++k) {
        v.cd_rot[k].V = v.Vr + (v.cd[k].V - v.V);
        v.cd_rot[k].d0 = v.eps0 + cd[k].eps_off;
    }
    v.rot_state = 1;
    return WPCD_OK;
}

// Allocate (or reuse) eigenpair storage for `S` samples of vset v and upload
// the channel table with this batch's offsets (a pageable host copy, so it
// stays outside CUDA graphs).
wpcd_status diag_prep(wpcd_ctx *c, Exec &X, VSetH &v, int vset_id, int S, int prec, EigH &e)
{
    size_t eps_len = 0, c_len = 0;
    std::vector<ChanDev> cd = v.cd;
    for (int k = 0; k < v.n_ch; ++k) {
        cd[k].eps_off = (long long)eps_len;
        cd[k].c_off = (long long)c_len;
        eps_len += (size_t)S * cd[k].n;
        c_len += (size_t)S * cd[k].n * cd[k].n;
    }
    const size_t coeff_len = (size_t)S * std::max(v.n_terms - 1, 1);
    wpcd_status st = WPCD_OK;
    // grow-only storage: a smaller batch or another set with as many channels reuses it
    if (e.eps_len < eps_len || e.c_len < c_len || e.coeff_len < coeff_len || e.status_len < (size_t)S * v.n_ch ||
        e.cd_len < (size_t)v.n_ch) {
        cudaStreamSynchronize(X.stream);
        free_eig(c, e);
        if ((st = dalloc(c, &e.eps, eps_len))) return st;
        if ((st = dalloc(c, &e.C, c_len))) return st;
        if ((st = dalloc(c, &e.coeffs, coeff_len))) return st;
        if ((st = dalloc(c, &e.status, (size_t)S * v.n_ch))) return st;
        if ((st = dalloc(c, &e.cd_dev, (size_t)v.n_ch))) return st;
        if ((st = dalloc(c, &e.cd_rot_dev, (size_t)v.n_ch))) return st;
        e.eps_len = eps_len;
        e.c_len = c_len;
        e.coeff_len = coeff_len;
        e.status_len = (size_t)S * v.n_ch;
        e.cd_len = (size_t)v.n_ch;
    }
    e.vset_id = vset_id;
    e.n_samples = S;
    e.prec = prec;
    CK(cudaMemcpyAsync(e.cd_dev, cd.data(), sizeof(ChanDev) * v.n_ch, cudaMemcpyHostToDevice, X.stream));
    e.rot = false;
    if (prec == WPCD_PREC_MIXED && c->rotate && c->refine_engine == WPCD_REFINE_TENSOR) {
        if ((st = ensure_rotation(c, X, v))) return st;
        if (v.rot_state == 1) {
            std::vector<ChanDev> cr = v.cd_rot;
            for (int k = 0; k < v.n_ch; ++k) {
                cr[k].eps_off = cd[k].eps_off;
                cr[k].c_off = cd[k].c_off;
            }
            CK(cudaMemcpyAsync(e.cd_rot_dev, cr.data(), sizeof(ChanDev) * v.n_ch, cudaMemcpyHostToDevice,
                               X.stream));
            e.rot = true;
        }
    }
    return WPCD_OK;
}

// A size bucket whose matrices exceed one CTA's shared memory: the Jacobi
// kernel with the matrix and eigenvectors in global memory (eig_big.cu), one
// scratch slot per resident CTA; the mixed path then refines as for the other
// sizes.
wpcd_status run_bucket_big(wpcd_ctx *c, Exec &X, VSetH &v, EigH &e, const double *cf, const int *work, int nw,
                           int nsmp, int smp0, int n, int prec)
{
    (void)v;
    const bool f64 = prec == WPCD_PREC_FP64;
    if (n > jacobi_big_max_n()) return WPCD_ERR_ARG;
    if (!c->n_sm) cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);
    const int occ = std::max(1, jacobi_big_occupancy(n, f64));
    const size_t slot_b = (jacobi_big_scratch_bytes(n, f64) + 255) & ~(size_t)255;
    // CTAs in flight: every resident one.  Each CTA's round is bound by the latency of
    // its L2 round trips, so the rate grows with the CTAs in flight (measured at
    // n = 512, FP32: 24 / 48 / 76 / 152 CTAs give 167 / 332 / 953 / 1518 solves/s)
    int cap = c->n_sm * occ;
    if (c->big_slots > 0) cap = c->big_slots;
    if (f64) {
        const int items = nsmp * nw;
        const int slots = std::max(1, std::min(items, cap));
        wpcd_status st = ws_reserve(c, X, X.ws_ref, slot_b * slots);
        if (st) return st;
        Launch L(c, X, WPCD_PHASE_EIGEN);
        CK(launch_jacobi_big(true, e.cd_dev, work, nw, nsmp, smp0, v.n_terms, cf, n, X.ws_ref.p, slots, e.eps, e.C,
                             nullptr, nullptr, nullptr, e.status, v.n_ch, X.err, X.stream));
        return WPCD_OK;
    }
    const size_t ref_item = refine_scratch_per_item(n, c->refine_engine);
    int chunk = (int)std::max<size_t>(1, kRefineScratchBytes / (ref_item * nw));
    chunk = std::min(chunk, std::max(1, 65535 / nw));  // the refinement grids put items in y / z (<= 65535)
    chunk = std::min(chunk, nsmp);
    const int slots = std::max(1, std::min(chunk * nw, cap));
    const size_t ref_b = (ref_item * nw * chunk + 255) & ~(size_t)255;
    wpcd_status st = ws_reserve(c, X, X.ws_ref, ref_b + slot_b * slots);
    if (st) return st;
    unsigned char *base = static_cast<unsigned char *>(X.ws_ref.p);
    double *Xs = reinterpret_cast<double *>(base);
    for (int s0 = 0; s0 < nsmp; s0 += chunk) {
        const int ns = std::min(chunk, nsmp - s0);
        {
            Launch L(c, X, WPCD_PHASE_EIGEN);
            // X, H and lambda in the layout of launch_refine (blocks 0, 1 and the lambda block)
            CK(launch_jacobi_big(false, e.rot ? e.cd_rot_dev : e.cd_dev, work, nw, ns, smp0 + s0, v.n_terms, cf, n,
                                 base + ref_b, slots, nullptr, nullptr, Xs + (size_t)5 * ns * nw * n * n, Xs,
                                 Xs + (size_t)ns * nw * n * n, e.status, v.n_ch, X.err, X.stream));
        }
        Launch L(c, X, WPCD_PHASE_REFINE);
        const VSetH::RotB *rb = e.rot ? &v.rotb.at(n) : nullptr;
        CK(launch_refine(e.cd_dev, work, nw, ns, smp0 + s0, n, v.n_terms, cf, base, e.eps, e.C, c->refine_iters,
                         c->refine_engine, X.stream, X.err, rb ? rb->sC : nullptr, rb ? rb->eC : nullptr, c->refine_digits));
    }
    return WPCD_OK;
}

// The parameter sum + eigensolve of the batch diag_prep set up (device-only
// work on X.stream: capturable).  coeffs: device, [S][n_terms - 1].
wpcd_status diag_body(wpcd_ctx *c, Exec &X, VSetH &v, const double *coeffs, int S, int prec, EigH &e)
{
    wpcd_status st = WPCD_OK;
    if (v.n_terms > 1) {
        CK(cudaMemcpyAsync(e.coeffs, coeffs, sizeof(double) * S * (v.n_terms - 1), cudaMemcpyDeviceToDevice,
                           X.stream));
    }
    const double *cf = v.n_terms > 1 ? e.coeffs : nullptr;
    // FP64: one Jacobi launch per size bucket (largest first), or per solve in plain mode.
    // MIXED: per bucket, in sample chunks sized to the refinement scratch, an FP32
    // Jacobi launch followed by two FP64 refinement iterations.
    auto run_bucket = [&](const int *work, int nw, int nsmp, int smp0, int n) -> wpcd_status {
        if (!jacobi_fits_smem(n, prec == WPCD_PREC_FP64)) return run_bucket_big(c, X, v, e, cf, work, nw, nsmp, smp0, n, prec);
        const int threads = pick_threads(c, X, n, prec, nw, nsmp, [&](int th, int ns) {
            if (prec == WPCD_PREC_FP64)
                return launch_jacobi_f64(e.cd_dev, work, nw, ns, smp0, v.n_terms, cf, n, e.eps, e.C, e.status, v.n_ch,
                                         X.err, X.stream, th);
            // the FP32 solve alone, into the start of the refinement scratch
            const bool cs = jacobi_mixed_c_in_smem(n);
            const size_t per = refine_scratch_per_item(n, c->refine_engine) + (cs ? 0 : jacobi_mixed_c_bytes(n)) + 256;
            if (ws_reserve(c, X, X.ws_ref, per * nw * ns)) return cudaErrorMemoryAllocation;
            unsigned char *base = static_cast<unsigned char *>(X.ws_ref.p);
            double *Xs = reinterpret_cast<double *>(base);
            const size_t c_off = (refine_scratch_per_item(n, c->refine_engine) * nw * ns + 255) & ~(size_t)255;
            return launch_jacobi_mixed(e.rot ? e.cd_rot_dev : e.cd_dev, work, nw, ns, smp0, v.n_terms, cf, n,
                                       Xs + (size_t)5 * ns * nw * n * n, Xs, reinterpret_cast<float *>(base + c_off),
                                       Xs + (size_t)ns * nw * n * n, e.status, v.n_ch, X.err, X.stream, th);
        });
        if (threads < 0) return WPCD_ERR_CUDA;
        if (prec == WPCD_PREC_FP64) {
            Launch L(c, X, WPCD_PHASE_EIGEN);
            CK(launch_jacobi_f64(e.cd_dev, work, nw, nsmp, smp0, v.n_terms, cf, n, e.eps, e.C, e.status, v.n_ch,
                                 X.err, X.stream, threads));
            return WPCD_OK;
        }
        const bool c_smem = jacobi_mixed_c_in_smem(n);
        const size_t ref_item = refine_scratch_per_item(n, c->refine_engine);
        const size_t per_item = ref_item + (c_smem ? 0 : jacobi_mixed_c_bytes(n)) + 256;
        int chunk = (int)std::max<size_t>(1, kRefineScratchBytes / (per_item * nw));
        chunk = std::min(chunk, std::max(1, 65535 / nw));  // the refinement grids put items in y / z (<= 65535)
        chunk = std::min(chunk, nsmp);
        wpcd_status st2 = ws_reserve(c, X, X.ws_ref, per_item * nw * chunk);
        if (st2) return st2;
        unsigned char *base = static_cast<unsigned char *>(X.ws_ref.p);
        double *Xs = reinterpret_cast<double *>(base);  // first block of the refinement scratch
        float *Cf = reinterpret_cast<float *>(base + ((ref_item * nw * chunk + 255) & ~(size_t)255));
        for (int s0 = 0; s0 < nsmp; s0 += chunk) {
            const int ns = std::min(chunk, nsmp - s0);
            {
                Launch L(c, X, WPCD_PHASE_EIGEN);
                // the FP64 H goes to the second n^2 block of the refinement scratch (layout of launch_refine)
                CK(launch_jacobi_mixed(e.rot ? e.cd_rot_dev : e.cd_dev, work, nw, ns, smp0 + s0, v.n_terms, cf, n,
                                       Xs + (size_t)5 * ns * nw * n * n, Xs, Cf, Xs + (size_t)ns * nw * n * n,
                                       e.status, v.n_ch, X.err, X.stream, threads));
            }
            Launch L(c, X, WPCD_PHASE_REFINE);
            const VSetH::RotB *rb = e.rot ? &v.rotb.at(n) : nullptr;
            CK(launch_refine(e.cd_dev, work, nw, ns, smp0 + s0, n, v.n_terms, cf, base, e.eps, e.C, c->refine_iters,
                             c->refine_engine, X.stream, X.err, rb ? rb->sC : nullptr, rb ? rb->eC : nullptr, c->refine_digits));
        }
        return WPCD_OK;
    };
    if (c->exec_mode == WPCD_EXEC_PLAIN) {
        // one solve per launch: the baseline execution on the same GPU
        for (int s = 0; s < S; ++s)
            for (int k = 0; k < v.n_ch; ++k)
                if ((st = run_bucket(v.ident_dev + k, 1, 1, s, v.cd[k].n))) return st;
    } else {
        for (auto it = v.buckets.rbegin(); it != v.buckets.rend(); ++it)
            if ((st = run_bucket(v.bucket_dev[it->first], (int)it->second.size(), S, 0, it->first))) return st;
    }
    return WPCD_OK;
}

wpcd_status run_diag(wpcd_ctx *c, Exec &X, VSetH &v, int vset_id, const double *coeffs, int S, int prec, EigH &e)
{
    wpcd_status st = diag_prep(c, X, v, vset_id, S, prec, e);
    return st ? st : diag_body(c, X, v, coeffs, S, prec, e);
}

// Energy plan + T at the needed bins into the executor's workspaces.  With
// n_E_s (device, per-sample list lengths) every sample has its own energy
// list at e_lab + s * n_E; otherwise one list serves all samples.
wpcd_status run_tbin(wpcd_ctx *c, Exec &X, VSetH &v, EigH &e, const double *e_lab, int n_E, const int *n_E_s,
                     PlanDev &plan, int res = WPCD_AVG_FREE_BIN)
{
    const int nch = v.n_ch, maxN = v.maxN, S = e.n_samples;
    const int P = n_E_s ? S : 1;
    wpcd_status st;
    const size_t ni = (size_t)P * (2 * (size_t)nch * n_E + nch + (size_t)nch * maxN);
    if ((st = ws_reserve(c, X, X.ws_plan_i, ni * sizeof(int)))) return st;
    if ((st = ws_reserve(c, X, X.ws_plan_d, (size_t)P * n_E * sizeof(double)))) return st;
    const size_t stride = res == WPCD_POINT ? (size_t)n_E : (size_t)maxN;  // items per (sample, channel)
    if ((st = ws_reserve(c, X, X.ws_tbin, (size_t)S * nch * stride * 8 * sizeof(double)))) return st;
    if ((st = ws_reserve(c, X, X.ws_phbin, (size_t)S * nch * stride * 3 * sizeof(double)))) return st;
    int *pi = static_cast<int *>(X.ws_plan_i.p);
    plan.bin = pi;
    plan.brk = pi + (size_t)P * nch * n_E;
    plan.cnt = plan.brk + (size_t)P * nch * n_E;
    plan.list = plan.cnt + (size_t)P * nch;
    plan.pE = static_cast<double *>(X.ws_plan_d.p);
    plan.per_sample = n_E_s ? 1 : 0;
    plan.n_E_s = n_E_s;
    plan.ip_frac = c->ip_frac;
    {
        Launch L(c, X, WPCD_PHASE_PLAN);
        CK(launch_plan(e.cd_dev, nch, maxN, e_lab, n_E, plan, X.err, X.stream, P));
    }
    Launch L(c, X, WPCD_PHASE_TMATRIX);
    const double *cf = v.n_terms > 1 ? e.coeffs : nullptr;
    double *tb = static_cast<double *>(X.ws_tbin.p), *pb = static_cast<double *>(X.ws_phbin.p);
    CK(launch_tbin(e.cd_dev, nch, S, v.n_terms, cf, e.eps, e.C, plan, maxN, n_E, tb, pb, X.err, X.stream,
                   e.prec == WPCD_PREC_MIXED, res));
    return WPCD_OK;
}

// T at the energies and/or phases + cross sections, after run_tbin.
wpcd_status run_outputs(wpcd_ctx *c, Exec &X, VSetH &v, EigH &e, int n_E, PlanDev &plan, double *t_out,
                        double *delta, double *sigma, int res = WPCD_AVG_FREE_BIN)
{
    const bool direct = res == WPCD_POINT;  // values at the energies themselves
    if (t_out) {
        Launch L(c, X, WPCD_PHASE_GATHER);
        CK(launch_gather_t(e.cd_dev, v.n_ch, e.n_samples, n_E, v.maxN, plan, static_cast<double *>(X.ws_tbin.p),
                           t_out, X.stream, direct));
    }
    if (delta || sigma) {
        Launch L(c, X, WPCD_PHASE_OBSERVABLES);
        CK(launch_observables(e.cd_dev, v.n_ch, e.n_samples, n_E, v.maxN, plan, static_cast<double *>(X.ws_phbin.p),
                              delta, sigma, X.stream, direct));
    }
    return WPCD_OK;
}

// A resolvent the vset supports: the SWP-bin average needs uncoupled channels.
bool resolvent_ok(const VSetH &v, int res)
{
    if (res == WPCD_AVG_FREE_BIN || res == WPCD_POINT) return true;
    if (res != WPCD_AVG_SWP_INDEX) return false;
    for (int k = 0; k < v.n_ch; ++k)
        if (v.cd[k].K != 1) return false;
    return true;
}

wpcd_status check_energies(const double *e_lab, int n_E)
{
    if (!e_lab || n_E < 1) return WPCD_ERR_ARG;
    return WPCD_OK;
}

}  // namespace

void serve_shutdown(wpcd_ctx *c);
bool serve_owns(wpcd_ctx *c, int id);

// ============================================================================================ ABI
extern "C" {

const char *wpcd_strerror(wpcd_status st)
{
    switch (st) {
    case WPCD_OK: return "ok";
    case WPCD_ERR_ARG: return "invalid argument";
    case WPCD_ERR_NOMEM: return "out of memory";
    case WPCD_ERR_BUDGET: return "HBM budget exceeded";
    case WPCD_ERR_NOCONVERGE: return "eigensolver did not converge";
    case WPCD_ERR_TIMEOUT: return "timeout";
    case WPCD_ERR_CUDA: return "CUDA error";
    case WPCD_ERR_NOTREADY: return "not ready";
    case WPCD_ERR_HANDLE: return "unknown handle";
    }
    return "unknown status";
}

wpcd_status wpcd_create(wpcd_ctx **out, int device, size_t hbm_budget_bytes, void *cuda_stream)
{
    if (!out) return WPCD_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return WPCD_ERR_ARG;
    }
    CK(cudaSetDevice(device));
    auto *c = new (std::nothrow) wpcd_ctx();
    if (!c) return WPCD_ERR_NOMEM;
    c->device = device;
    c->main.stream = static_cast<cudaStream_t>(cuda_stream);
    c->budget = hbm_budget_bytes;
    if (dalloc(c, &c->err_dev, 1) != WPCD_OK || cudaMemsetAsync(c->err_dev, 0, sizeof(int), c->main.stream) != cudaSuccess) {
        delete c;
        return WPCD_ERR_CUDA;
    }
    c->main.err = c->err_dev;
    *out = c;
    return WPCD_OK;
}

void wpcd_destroy(wpcd_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->main.stream);
    for (auto &kv : c->handles) {
        if (kv.second.mesh) free_mesh(c, *kv.second.mesh);
        if (kv.second.vset) free_vset(c, *kv.second.vset);
        if (kv.second.eig) free_eig(c, *kv.second.eig);
        if (kv.second.mi) free_mi(c, *kv.second.mi);
    }
    serve_shutdown(c);
    for (auto &kv : c->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    c->graphs.clear();
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    free_eig(c, c->main.eig);
    for (auto &kv : c->gl) {
        dfree(c, kv.second.first);
        dfree(c, kv.second.second);
    }
    Exec &M = c->main;
    for (auto *b : {&M.ws_plan_i, &M.ws_plan_d, &M.ws_tbin, &M.ws_phbin, &M.ws_in, &M.ws_out, &M.ws_ref}) dfree(c, b->p);
    dfree(c, c->err_dev);
    delete c;
}

wpcd_status wpcd_set_option(wpcd_ctx *c, int key, int value)
{
    if (!c) return WPCD_ERR_ARG;
    ++c->graph_gen;  // any option may change what a graph baked in
    if (key == WPCD_OPT_GRAPH && (value == 0 || value == 1)) {
        c->use_graphs = value;
        return WPCD_OK;
    }
    if (key == WPCD_OPT_EXEC && (value == WPCD_EXEC_BATCHED || value == WPCD_EXEC_PLAIN)) {
        c->exec_mode = value;
        return WPCD_OK;
    }
    if (key == WPCD_OPT_REFINE && (value == WPCD_REFINE_TENSOR || value == WPCD_REFINE_FP64)) {
        c->refine_engine = value;
        return WPCD_OK;
    }
    if (key == WPCD_OPT_REFINE_ITERS && value >= 1 && value <= 4) {
        c->refine_iters = value;
        return WPCD_OK;
    }
    if (key == WPCD_OPT_REFINE_DIGITS && value >= 4 && value <= 6) {
        c->refine_digits = value;
        return WPCD_OK;
    }
    if (key == WPCD_OPT_ROTATE && (value == 0 || value == 1)) {
        c->rotate = value;
        return WPCD_OK;
    }
    if (key == WPCD_OPT_BIG_SLOTS && value >= 0) {
        c->big_slots = value;
        return WPCD_OK;
    }
    if (key == WPCD_OPT_AUTOTUNE && (value == 0 || value == 1)) {
        c->autotune = value;
        if (!value) {
            std::lock_guard<std::mutex> lk(c->tmu);
            c->tuned.clear();
        }
        return WPCD_OK;
    }
    return WPCD_ERR_ARG;
}

wpcd_status wpcd_set_interp_point(wpcd_ctx *c, double frac)
{
    if (!c || !(frac > 0.0 && frac < 1.0)) return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    c->ip_frac = frac;
    ++c->graph_gen;  // captured graphs hold the energy plan's value
    return WPCD_OK;
}

wpcd_status wpcd_sync(wpcd_ctx *c)
{
    if (!c) return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    CK(cudaSetDevice(c->device));
    int h = 0;
    CK(cudaMemcpyAsync(&h, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost, c->main.stream));
    CK(cudaStreamSynchronize(c->main.stream));
    if (h != 0) CK(cudaMemsetAsync(c->err_dev, 0, sizeof(int), c->main.stream));
    switch (h) {
    case kDevOk: return WPCD_OK;
    case kDevEnergyOutside: return WPCD_ERR_ARG;
    case kDevMode: return WPCD_ERR_ARG;
    case kDevTimeout: return WPCD_ERR_TIMEOUT;
    case kDevNoConverge: return WPCD_ERR_NOCONVERGE;
    case kDevBadSize: return WPCD_ERR_CUDA;
    default: return WPCD_ERR_ARG;
    }
}

size_t wpcd_bytes_in_use(const wpcd_ctx *c) { return c ? c->in_use : 0; }

wpcd_status wpcd_mesh(wpcd_ctx *c, int n_wp, int kind, double alpha, double t, double kmax, int n_quad, int wp_kind,
                      int *mesh_id)
{
    if (!c || !mesh_id || n_wp < 4 || n_wp > kMaxNwp || n_quad < 1 || n_quad > kMaxQ || !(alpha > 0) || !(t > 0) ||
        (kind != 0 && kind != 1) || (wp_kind != 0 && wp_kind != 1) || (kind == 0 && !(kmax > 0)))
        return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    CK(cudaSetDevice(c->device));
    auto m = std::make_unique<MeshH>();
    m->N = n_wp;
    m->Q = n_quad;
    m->kind = kind;
    m->wp_kind = wp_kind;
    m->alpha = alpha;
    m->t = t;
    m->kmax = kmax;
    wpcd_status st;
    double *glx, *glw;
    if ((st = gl_rule(c, n_quad, &glx, &glw))) return st;
    if ((st = dalloc(c, &m->kb, n_wp + 1)) || (st = dalloc(c, &m->kq, (size_t)n_wp * n_quad)) ||
        (st = dalloc(c, &m->wq, (size_t)n_wp * n_quad)) || (st = dalloc(c, &m->h0, n_wp))) {
        free_mesh(c, *m);
        return st;
    }
    Launch L(c, c->main, WPCD_PHASE_MESH);
    CK(launch_mesh(n_wp, kind, alpha, t, kmax, n_quad, wp_kind, glx, glw, m->kb, m->kq, m->wq, m->h0, c->main.stream));
    int id = c->next_id++;
    Handle h;
    h.kind = kMesh;
    h.mesh = std::move(m);
    c->handles.emplace(id, std::move(h));
    *mesh_id = id;
    return WPCD_OK;
}

wpcd_status wpcd_mesh_get(wpcd_ctx *c, int mesh_id, double *kb, double *kq, double *wq)
{
    if (!c) return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    Handle *h = find(c, mesh_id, kMesh);
    if (!h) return WPCD_ERR_HANDLE;
    CK(cudaSetDevice(c->device));
    MeshH &m = *h->mesh;
    if (kb) CK(cudaMemcpyAsync(kb, m.kb, sizeof(double) * (m.N + 1), cudaMemcpyDeviceToHost, c->main.stream));
    if (kq) CK(cudaMemcpyAsync(kq, m.kq, sizeof(double) * m.N * m.Q, cudaMemcpyDeviceToHost, c->main.stream));
    if (wq) CK(cudaMemcpyAsync(wq, m.wq, sizeof(double) * m.N * m.Q, cudaMemcpyDeviceToHost, c->main.stream));
    CK(cudaStreamSynchronize(c->main.stream));
    return WPCD_OK;
}

wpcd_status wpcd_project(wpcd_ctx *c, const int *mesh_ids, const wpcd_channel *chs, int n_ch, int gen,
                         const double *gp_host, int n_gp, const double *v_fine_dev, int n_terms, int *vset_id)
{
    return wpcd_project_prec(c, mesh_ids, chs, n_ch, gen, gp_host, n_gp, v_fine_dev, n_terms, WPCD_PREC_FP64, vset_id);
}

wpcd_status wpcd_project_prec(wpcd_ctx *c, const int *mesh_ids, const wpcd_channel *chs, int n_ch, int gen,
                              const double *gp_host, int n_gp, const double *v_fine_dev, int n_terms,
                              wpcd_precision prec, int *vset_id)
{
    if (!c || !mesh_ids || !chs || n_ch < 1 || !vset_id || n_terms < 1 || n_terms > kMaxTerms) return WPCD_ERR_ARG;
    if (prec != WPCD_PREC_FP64 && prec != WPCD_PREC_MIXED) return WPCD_ERR_ARG;
    if (gen == WPCD_GEN_YAMAGUCHI && (n_terms != 1 || !gp_host || n_gp < 2)) return WPCD_ERR_ARG;
    if (gen == WPCD_GEN_YUKAWA && (n_terms > kYukTerms + 1 || !gp_host || n_gp < kYukParams)) return WPCD_ERR_ARG;
    if (gen == WPCD_GEN_FINE && !v_fine_dev) return WPCD_ERR_ARG;
    if (gen != WPCD_GEN_FINE && gen != WPCD_GEN_YAMAGUCHI && gen != WPCD_GEN_YUKAWA) return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    CK(cudaSetDevice(c->device));
    auto v = std::make_unique<VSetH>();
    v->n_ch = n_ch;
    v->n_terms = n_terms;
    v->gen = gen;
    size_t vlen = 0;
    int maxJ = 0;
    for (int k = 0; k < n_ch; ++k) {
        const wpcd_channel &ch = chs[k];
        Handle *h = find(c, mesh_ids[k], kMesh);
        if (!h) return WPCD_ERR_HANDLE;
        if (ch.J < 0 || ch.J > kMaxJ || (ch.s != 0 && ch.s != 1)) return WPCD_ERR_ARG;
        if (ch.coupled && (ch.s != 1 || ch.J < 1 || ch.l != ch.J - 1 || ch.lp != ch.J + 1)) return WPCD_ERR_ARG;
        if (!ch.coupled && ch.l != ch.lp) return WPCD_ERR_ARG;
        if (gen == WPCD_GEN_YAMAGUCHI && (ch.coupled || ch.l != 0)) return WPCD_ERR_ARG;
        if (gen == WPCD_GEN_YUKAWA && ch.J > 8) return WPCD_ERR_ARG;
        MeshH &m = *h->mesh;
        ChanDev d;
        memset(&d, 0, sizeof(d));
        d.s = ch.s;
        d.J = ch.J;
        d.l = ch.l;
        d.lp = ch.lp;
        d.coupled = ch.coupled ? 1 : 0;
        d.tz = ch.tz;
        d.N = m.N;
        d.K = ch.coupled ? 2 : 1;
        d.n = d.K * m.N;
        d.Q = m.Q;
        d.wp_kind = m.wp_kind;
        d.kb = m.kb;
        d.kq = m.kq;
        d.wq = m.wq;
        d.h0 = m.h0;
        d.eps_off = (long long)vlen;  // temporarily: offset of V
        vlen += (size_t)n_terms * d.n * d.n;
        v->cd.push_back(d);
        v->ch.push_back(ch);
        v->mesh_ids.push_back(mesh_ids[k]);
        v->maxN = std::max(v->maxN, m.N);
        v->maxn = std::max(v->maxn, d.n);
        maxJ = std::max(maxJ, ch.J);
    }
    wpcd_status st;
    if ((st = dalloc(c, &v->V, vlen))) return st;
    for (auto &d : v->cd) {
        d.V = v->V + d.eps_off;
        d.eps_off = 0;
    }
    if ((st = dalloc(c, &v->cd_dev, (size_t)n_ch)) || (st = dalloc(c, &v->ident_dev, (size_t)n_ch))) {
        free_vset(c, *v);
        return st;
    }
    std::vector<int> ident(n_ch);
    for (int k = 0; k < n_ch; ++k) {
        ident[k] = k;
        v->buckets[v->cd[k].n].push_back(k);
    }
    CK(cudaMemcpyAsync(v->cd_dev, v->cd.data(), sizeof(ChanDev) * n_ch, cudaMemcpyHostToDevice, c->main.stream));
    CK(cudaMemcpyAsync(v->ident_dev, ident.data(), sizeof(int) * n_ch, cudaMemcpyHostToDevice, c->main.stream));
    for (auto &kv : v->buckets) {
        int *p;
        if ((st = dalloc(c, &p, kv.second.size()))) {
            free_vset(c, *v);
            return st;
        }
        v->bucket_dev[kv.first] = p;
        CK(cudaMemcpyAsync(p, kv.second.data(), sizeof(int) * kv.second.size(), cudaMemcpyHostToDevice, c->main.stream));
    }
    if (gen == WPCD_GEN_FINE) {
        size_t off = 0;
        for (int k = 0; k < n_ch; ++k) {
            const ChanDev &d = v->cd[k];
            Launch L(c, c->main, WPCD_PHASE_PROJECT);
            CK(launch_project_fine(v->cd_dev, k, d, v_fine_dev + off, n_terms, c->main.stream));
            const size_t knq = (size_t)d.K * d.N * d.Q;
            off += (size_t)n_terms * knq * knq;
        }
    } else {
        // parameters to the device (a small transient buffer, freed after the stream drains)
        double *gp_dev;
        if ((st = dalloc(c, &gp_dev, (size_t)n_gp))) {
            free_vset(c, *v);
            return st;
        }
        CK(cudaMemcpyAsync(gp_dev, gp_host, sizeof(double) * n_gp, cudaMemcpyHostToDevice, c->main.stream));
        double *angx = nullptr, *angw = nullptr;
        if (gen == WPCD_GEN_YUKAWA && (st = gl_rule(c, kAngleQ, &angx, &angw))) return st;
        // group the channels by mesh; one launch per mesh
        std::map<int, std::vector<int>> groups;
        for (int k = 0; k < n_ch; ++k) groups[mesh_ids[k]].push_back(k);
        std::vector<int *> gdevs;
        std::vector<float *> gdevs_f;  // angle-integral buffers of the reduced-precision projection
        for (auto &kv : groups) {
            int *gd;
            if ((st = dalloc(c, &gd, kv.second.size()))) return st;
            gdevs.push_back(gd);
            CK(cudaMemcpyAsync(gd, kv.second.data(), sizeof(int) * kv.second.size(), cudaMemcpyHostToDevice,
                               c->main.stream));
            const ChanDev &d0 = v->cd[kv.second[0]];
            Launch L(c, c->main, WPCD_PHASE_PROJECT);
            if (gen == WPCD_GEN_YUKAWA) {
                // reduced precision: the angle integrals from the tensor-core contraction
                float *Ibuf = nullptr;
                if (prec == WPCD_PREC_MIXED) {
                    if ((st = dmalloc(c, reinterpret_cast<void **>(&Ibuf), angle_tc_buffer_bytes(d0.N, d0.Q)))) return st;
                    gdevs_f.push_back(Ibuf);
                    CK(launch_angle_tc(v->cd_dev, gd, d0.N, d0.Q, maxJ + 2, gp_dev, angx, angw, Ibuf, c->main.err,
                                       c->main.stream));
                }
                CK(launch_project_yukawa(v->cd_dev, gd, (int)kv.second.size(), d0.N, d0.Q, maxJ + 2, gp_dev, angx, angw,
                                         n_terms, c->main.stream, Ibuf));
            } else
                CK(launch_project_yamaguchi_gp(v->cd_dev, gd, (int)kv.second.size(), d0.N, d0.Q, gp_dev, c->main.stream));
        }
        CK(cudaStreamSynchronize(c->main.stream));
        for (int *gd : gdevs) dfree(c, gd);
        for (float *fb : gdevs_f) dfree(c, fb);
        dfree(c, gp_dev);
    }
    int id = c->next_id++;
    Handle h;
    h.kind = kVSet;
    h.vset = std::move(v);
    c->handles.emplace(id, std::move(h));
    *vset_id = id;
    return WPCD_OK;
}

wpcd_status wpcd_vset_info(wpcd_ctx *c, int vset_id, int *n_ch, int *n_terms, int channel, int *n)
{
    if (!c) return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    Handle *h = find(c, vset_id, kVSet);
    if (!h) return WPCD_ERR_HANDLE;
    VSetH &v = *h->vset;
    if (n_ch) *n_ch = v.n_ch;
    if (n_terms) *n_terms = v.n_terms;
    if (n) {
        if (channel < 0 || channel >= v.n_ch) return WPCD_ERR_ARG;
        *n = v.cd[channel].n;
    }
    return WPCD_OK;
}

wpcd_status wpcd_vset_get(wpcd_ctx *c, int vset_id, int channel, double *out)
{
    if (!c || !out) return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    Handle *h = find(c, vset_id, kVSet);
    if (!h) return WPCD_ERR_HANDLE;
    VSetH &v = *h->vset;
    if (channel < 0 || channel >= v.n_ch) return WPCD_ERR_ARG;
    CK(cudaSetDevice(c->device));
    const ChanDev &d = v.cd[channel];
    CK(cudaMemcpyAsync(out, d.V, sizeof(double) * v.n_terms * d.n * d.n, cudaMemcpyDeviceToHost, c->main.stream));
    CK(cudaStreamSynchronize(c->main.stream));
    return WPCD_OK;
}

wpcd_status wpcd_diag(wpcd_ctx *c, int vset_id, const double *coeffs_dev, int n_samples, wpcd_precision prec,
                      int *eig_id)
{
    if (!c || !eig_id || n_samples < 1 || (prec != WPCD_PREC_FP64 && prec != WPCD_PREC_MIXED)) return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    Handle *h = find(c, vset_id, kVSet);
    if (!h) return WPCD_ERR_HANDLE;
    VSetH &v = *h->vset;
    if (v.n_terms > 1 && !coeffs_dev) return WPCD_ERR_ARG;
    CK(cudaSetDevice(c->device));
    auto e = std::make_unique<EigH>();
    wpcd_status st = run_diag(c, c->main, v, vset_id, coeffs_dev, n_samples, prec, *e);
    if (st) {
        free_eig(c, *e);
        return st;
    }
    int id = c->next_id++;
    Handle hh;
    hh.kind = kEig;
    hh.eig = std::move(e);
    c->handles.emplace(id, std::move(hh));
    *eig_id = id;
    return WPCD_OK;
}

wpcd_status wpcd_diag_status(wpcd_ctx *c, int eig_id, int *status_dev)
{
    if (!c || !status_dev) return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    Handle *h = find(c, eig_id, kEig);
    if (!h) return WPCD_ERR_HANDLE;
    EigH &e = *h->eig;
    Handle *hv = find(c, e.vset_id, kVSet);
    if (!hv) return WPCD_ERR_HANDLE;
    CK(cudaSetDevice(c->device));
    CK(cudaMemcpyAsync(status_dev, e.status, sizeof(int) * e.n_samples * hv->vset->n_ch, cudaMemcpyDeviceToDevice,
                       c->main.stream));
    return WPCD_OK;
}

wpcd_status wpcd_eig_get(wpcd_ctx *c, int eig_id, int sample, int channel, double *eps_host, double *C_host)
{
    if (!c) return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    Handle *h = find(c, eig_id, kEig);
    if (!h) return WPCD_ERR_HANDLE;
    EigH &e = *h->eig;
    Handle *hv = find(c, e.vset_id, kVSet);
    if (!hv) return WPCD_ERR_HANDLE;
    VSetH &v = *hv->vset;
    if (sample < 0 || sample >= e.n_samples || channel < 0 || channel >= v.n_ch) return WPCD_ERR_ARG;
    CK(cudaSetDevice(c->device));
    size_t eo = 0, co = 0;
    for (int k = 0; k < channel; ++k) {
        eo += (size_t)e.n_samples * v.cd[k].n;
        co += (size_t)e.n_samples * v.cd[k].n * v.cd[k].n;
    }
    const int n = v.cd[channel].n;
    if (eps_host)
        CK(cudaMemcpyAsync(eps_host, e.eps + eo + (size_t)sample * n, sizeof(double) * n, cudaMemcpyDeviceToHost,
                           c->main.stream));
    if (C_host)
        CK(cudaMemcpyAsync(C_host, e.C + co + (size_t)sample * n * n, sizeof(double) * n * n, cudaMemcpyDeviceToHost,
                           c->main.stream));
    CK(cudaStreamSynchronize(c->main.stream));
    return WPCD_OK;
}

static wpcd_status tmatrix_impl(wpcd_ctx *c, VSetH &v, EigH &e, const double *e_lab, int n_E, int res,
                                double *t_out, double *delta, double *sigma)
{
    if (!resolvent_ok(v, res)) return WPCD_ERR_ARG;
    PlanDev plan{};
    wpcd_status st = run_tbin(c, c->main, v, e, e_lab, n_E, nullptr, plan, res);
    if (st) return st;
    return run_outputs(c, c->main, v, e, n_E, plan, t_out, delta, sigma, res);
}

wpcd_status wpcd_tmatrix(wpcd_ctx *c, int eig_id, const double *e_lab, int n_E, wpcd_resolvent res, double *t_out)
{
    if (!c || !t_out || check_energies(e_lab, n_E)) return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    Handle *h = find(c, eig_id, kEig);
    if (!h) return WPCD_ERR_HANDLE;
    Handle *hv = find(c, h->eig->vset_id, kVSet);
    if (!hv) return WPCD_ERR_HANDLE;
    CK(cudaSetDevice(c->device));
    return tmatrix_impl(c, *hv->vset, *h->eig, e_lab, n_E, res, t_out, nullptr, nullptr);
}

wpcd_status wpcd_observables_res(wpcd_ctx *c, int eig_id, const double *e_lab, int n_E, wpcd_resolvent res,
                                 double *delta, double *sigma)
{
    if (!c || check_energies(e_lab, n_E) || (!delta && !sigma)) return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    Handle *h = find(c, eig_id, kEig);
    if (!h) return WPCD_ERR_HANDLE;
    Handle *hv = find(c, h->eig->vset_id, kVSet);
    if (!hv) return WPCD_ERR_HANDLE;
    CK(cudaSetDevice(c->device));
    return tmatrix_impl(c, *hv->vset, *h->eig, e_lab, n_E, res, nullptr, delta, sigma);
}

wpcd_status wpcd_observables(wpcd_ctx *c, int eig_id, const double *e_lab, int n_E, double *delta, double *sigma)
{
    return wpcd_observables_res(c, eig_id, e_lab, n_E, WPCD_AVG_FREE_BIN, delta, sigma);
}

// wpcd_solve through the graph cache (the caller holds c->mu).  First sight of
// a key: launch one by one and remember the key under the current generation.
// Second sight under the same generation: capture the device work on the
// private stream, instantiate, launch.  Later: launch the graph.  The channel
// table upload (diag_prep) runs before every launch, outside the graph.
static wpcd_status solve_graph(wpcd_ctx *c, VSetH &v, int vset_id, const double *coeffs, int S, const double *e_lab,
                               int n_E, int prec, int res, double *t_out, double *delta, double *sigma)
{
    Exec &X = c->main;
    EigH &e = X.eig;
    auto body = [&]() -> wpcd_status {
        wpcd_status st = diag_body(c, X, v, coeffs, S, prec, e);
        return st ? st : tmatrix_impl(c, v, e, e_lab, n_E, res, t_out, delta, sigma);
    };
    typedef unsigned long long u64;
    const std::array<u64, 12> key = {(u64)vset_id, (u64)S, (u64)n_E, (u64)prec, (u64)res, (u64)c->refine_engine,
                                     (u64)(uintptr_t)coeffs, (u64)(uintptr_t)e_lab, (u64)(uintptr_t)t_out,
                                     (u64)(uintptr_t)delta, (u64)(uintptr_t)sigma, (u64)(uintptr_t)X.stream};
    auto drop = [&](std::map<std::array<u64, 12>, wpcd_ctx::GraphE>::iterator it) {
        if (it->second.exec) cudaGraphExecDestroy(it->second.exec);
        c->graphs.erase(it);
    };
    auto it = c->graphs.find(key);
    if (it != c->graphs.end() && it->second.gen != c->graph_gen.load()) {
        drop(it);
        it = c->graphs.end();
    }
    wpcd_status st = diag_prep(c, X, v, vset_id, S, prec, e);
    if (st) return st;
    if (it == c->graphs.end() || it->second.failed) {
        if ((st = body())) return st;
        if (it == c->graphs.end()) {
            if (c->graphs.size() >= kGraphCache) {  // forget keys seen once, then everything
                for (auto jt = c->graphs.begin(); jt != c->graphs.end();)
                    jt = jt->second.exec ? std::next(jt) : c->graphs.erase(jt);
                while (c->graphs.size() >= kGraphCache) drop(c->graphs.begin());
            }
            c->graphs[key].gen = c->graph_gen.load();
        }
        return WPCD_OK;
    }
    wpcd_ctx::GraphE &g = it->second;
    if (g.gen != c->graph_gen.load()) {  // diag_prep reallocated the eigenpair storage
        drop(it);
        return body();
    }
    if (!g.exec) {
        if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        cudaStream_t user = X.stream;
        const u64 k0 = g_thread_kernels;
        cudaGraph_t graph = nullptr;
        wpcd_status cst = WPCD_ERR_CUDA;
        X.stream = c->cap_stream;
        if (cudaStreamBeginCapture(X.stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            cst = body();
            if (cudaStreamEndCapture(X.stream, &graph) != cudaSuccess) cst = WPCD_ERR_CUDA;
        }
        X.stream = user;
        const u64 kernels = g_thread_kernels - k0;
        c->launches -= kernels;  // captured, not launched
        cudaGraphExec_t exec = nullptr;
        if (cst == WPCD_OK && graph && g.gen == c->graph_gen.load() &&
            cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
            exec = nullptr;
        if (graph) cudaGraphDestroy(graph);
        if (!exec) {  // not capturable: this key stays one by one
            cudaGetLastError();
            g.failed = true;
            return body();
        }
        g.exec = exec;
        g.kernels = kernels;
        ++c->graph_captures;
    }
    CK(cudaGraphLaunch(g.exec, X.stream));
    c->launches += g.kernels;
    ++c->graph_replays;
    return WPCD_OK;
}

wpcd_status wpcd_solve(wpcd_ctx *c, int vset_id, const double *coeffs, int S, const double *e_lab, int n_E,
                       wpcd_precision prec, wpcd_resolvent res, double *t_out, double *delta, double *sigma)
{
    if (!c || S < 1 || (prec != WPCD_PREC_FP64 && prec != WPCD_PREC_MIXED) || check_energies(e_lab, n_E))
        return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    Handle *hv = find(c, vset_id, kVSet);
    if (!hv) return WPCD_ERR_HANDLE;
    VSetH &v = *hv->vset;
    if (v.n_terms > 1 && !coeffs) return WPCD_ERR_ARG;
    if (!resolvent_ok(v, res)) return WPCD_ERR_ARG;
    CK(cudaSetDevice(c->device));
    if (c->use_graphs && c->exec_mode == WPCD_EXEC_BATCHED && !c->prof)
        return solve_graph(c, v, vset_id, coeffs, S, e_lab, n_E, prec, res, t_out, delta, sigma);
    wpcd_status st = run_diag(c, c->main, v, vset_id, coeffs, S, prec, c->main.eig);
    if (st) return st;
    return tmatrix_impl(c, v, c->main.eig, e_lab, n_E, res, t_out, delta, sigma);
}

wpcd_status wpcd_solve_host(wpcd_ctx *c, int vset_id, const double *coeffs_h, int S, const double *e_lab_h, int n_E,
                            wpcd_precision prec, wpcd_resolvent res, double *t_h, double *delta_h, double *sigma_h)
{
    if (!c || S < 1 || !e_lab_h || n_E < 1) return WPCD_ERR_ARG;
    int n_ch = 0, n_terms = 0;
    wpcd_status st = wpcd_vset_info(c, vset_id, &n_ch, &n_terms, 0, nullptr);
    if (st) return st;
    if (n_terms > 1 && !coeffs_h) return WPCD_ERR_ARG;
    const size_t nc = n_terms > 1 ? (size_t)S * (n_terms - 1) : 0;
    const size_t in_bytes = (nc + n_E) * sizeof(double);
    const size_t nt = t_h ? (size_t)S * n_ch * n_E * 8 : 0, nd = delta_h ? (size_t)S * n_ch * n_E * 3 : 0,
                 ns = sigma_h ? (size_t)S * n_E : 0;
    const size_t out_bytes = (nt + nd + ns) * sizeof(double);
    double *din, *dout;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        CK(cudaSetDevice(c->device));
        if ((st = ws_reserve(c, c->main, c->main.ws_in, in_bytes)) || (st = ws_reserve(c, c->main, c->main.ws_out, out_bytes))) return st;
        din = static_cast<double *>(c->main.ws_in.p);
        dout = static_cast<double *>(c->main.ws_out.p);
        // straight from and into the caller's buffers: a host-to-device copy from
        // pageable memory returns once the source has been consumed, and the
        // device-to-host copies below are waited for before this call returns
        if (nc) CK(cudaMemcpyAsync(din, coeffs_h, nc * sizeof(double), cudaMemcpyHostToDevice, c->main.stream));
        CK(cudaMemcpyAsync(din + nc, e_lab_h, n_E * sizeof(double), cudaMemcpyHostToDevice, c->main.stream));
    }
    st = wpcd_solve(c, vset_id, nc ? din : nullptr, S, din + nc, n_E, prec, res, t_h ? dout : nullptr,
                    delta_h ? dout + nt : nullptr, sigma_h ? dout + nt + nd : nullptr);
    if (st) return st;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        if (t_h) CK(cudaMemcpyAsync(t_h, dout, nt * sizeof(double), cudaMemcpyDeviceToHost, c->main.stream));
        if (delta_h)
            CK(cudaMemcpyAsync(delta_h, dout + nt, nd * sizeof(double), cudaMemcpyDeviceToHost, c->main.stream));
        if (sigma_h)
            CK(cudaMemcpyAsync(sigma_h, dout + nt + nd, ns * sizeof(double), cudaMemcpyDeviceToHost,
                               c->main.stream));
    }
    st = wpcd_sync(c);
    return st;
}

wpcd_status wpcd_batched_dgemm(wpcd_ctx *c, int n, int items, int trans_a, const double *A_dev, const double *B_dev,
                                double *C_dev, int engine)
{
    if (!c || n < 1 || n > 2 * kMaxNwp || items < 1 || !A_dev || !B_dev || !C_dev ||
        (engine != WPCD_REFINE_TENSOR && engine != WPCD_REFINE_FP64))
        return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    CK(cudaSetDevice(c->device));
    wpcd_status st = ws_reserve(c, c->main, c->main.ws_ref, batched_dgemm_scratch(n, items));
    if (st) return st;
    Launch L(c, c->main, WPCD_PHASE_REFINE);
    CK(launch_batched_dgemm(n, items, trans_a != 0, A_dev, B_dev, C_dev, c->main.ws_ref.p, engine, c->main.stream,
                            c->main.err));
    return WPCD_OK;
}

int wpcd_tuning(wpcd_ctx *c, int max_entries, int *n_out, int *prec_out, int *threads_out, float *ms_out)
{
    if (!c) return 0;
    std::lock_guard<std::mutex> lk(c->tmu);
    int k = 0;
    for (auto &kv : c->tuned) {
        if (k >= max_entries) break;
        if (n_out) n_out[k] = kv.first.first;
        if (prec_out) prec_out[k] = kv.first.second;
        if (threads_out) threads_out[k] = kv.second.threads;
        if (ms_out)
            for (int j = 0; j < 5; ++j) ms_out[5 * k + j] = kv.second.ms[j];
        ++k;
    }
    return k;
}

unsigned long long wpcd_kernel_launches(const wpcd_ctx *c) { return c ? c->launches.load() : 0ULL; }

wpcd_status wpcd_device_log(wpcd_ctx *c, const double *x_dev, double *y_dev, int n)
{
    if (!c || n < 0 || (n > 0 && (!x_dev || !y_dev))) return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    CK(cudaSetDevice(c->device));
    Launch L(c, c->main, WPCD_PHASE_TMATRIX);
    CK(launch_wlog(x_dev, y_dev, n, c->main.stream));
    return WPCD_OK;
}

wpcd_status wpcd_graph_stats(wpcd_ctx *c, unsigned long long *captures, unsigned long long *replays, int *cached)
{
    if (!c) return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    if (captures) *captures = c->graph_captures;
    if (replays) *replays = c->graph_replays;
    if (cached) {
        int k = 0;
        for (auto &kv : c->graphs) k += kv.second.exec != nullptr;
        *cached = k;
    }
    return WPCD_OK;
}

wpcd_status wpcd_profile(wpcd_ctx *c, int enable)
{
    if (!c) return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    CK(cudaSetDevice(c->device));
    prof_collect(c);
    for (int k = 0; k < WPCD_PHASE_COUNT; ++k) {
        c->prof_ms[k] = 0.0;
        c->prof_n[k] = 0;
    }
    c->prof = enable != 0;
    return WPCD_OK;
}

wpcd_status wpcd_profile_read(wpcd_ctx *c, int phase, double *ms_total, long *launches)
{
    if (!c || phase < 0 || phase >= WPCD_PHASE_COUNT) return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    CK(cudaSetDevice(c->device));
    prof_collect(c);
    if (ms_total) *ms_total = c->prof_ms[phase];
    if (launches) *launches = c->prof_n[phase];
    return WPCD_OK;
}

wpcd_status wpcd_release(wpcd_ctx *c, int id)
{
    if (!c) return WPCD_ERR_ARG;
    if (serve_owns(c, id)) return WPCD_ERR_ARG;  // meshes and sets of a running server stay
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->handles.find(id);
    if (it == c->handles.end()) return WPCD_ERR_HANDLE;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->main.stream);
    if (it->second.mesh) free_mesh(c, *it->second.mesh);
    if (it->second.vset) free_vset(c, *it->second.vset);
    if (it->second.eig) free_eig(c, *it->second.eig);
    if (it->second.mi) free_mi(c, *it->second.mi);
    c->handles.erase(it);
    return WPCD_OK;
}

// ---- spin observables (App. A) ---------------------------------------------------------------------
namespace {
// Clebsch-Gordan <j1 m1 j2 m2 | J M> for integer spins, Racah's closed form.
double cg_racah(int j1, int m1, int j2, int m2, int J, int M)
{
    if (m1 + m2 != M || std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(M) > J || J < std::abs(j1 - j2) ||
        J > j1 + j2)
        return 0.0;
    auto lf = [](int n) { return std::lgamma((double)n + 1.0); };
    const double pre = 0.5 * (std::log(2.0 * J + 1.0) + lf(J + j1 - j2) + lf(J - j1 + j2) + lf(j1 + j2 - J) -
                              lf(j1 + j2 + J + 1) + lf(J + M) + lf(J - M) + lf(j1 - m1) + lf(j1 + m1) + lf(j2 - m2) +
                              lf(j2 + m2));
    double sum = 0.0;
    for (int k = 0; k <= j1 + j2 - J; ++k) {
        const int a = j1 + j2 - J - k, b = j1 - m1 - k, c = j2 + m2 - k, d = J - j2 + m1 + k, e = J - j1 - m2 + k;
        if (a < 0 || b < 0 || c < 0 || d < 0 || e < 0) continue;
        const double t = std::exp(pre - lf(k) - lf(a) - lf(b) - lf(c) - lf(d) - lf(e));
        sum += (k & 1) ? -t : t;
    }
    return sum;
}
}  // namespace

wpcd_status wpcd_saclay(wpcd_ctx *c, const wpcd_channel *channels, int n_ch, const double *delta, int S,
                        const double *e_lab, int n_E, const double *theta, int n_theta, double *abcde, double *dsig)
{
    if (!c || !channels || n_ch < 1 || !delta || S < 1 || !e_lab || n_E < 1 || !theta || n_theta < 1 ||
        (!abcde && !dsig))
        return WPCD_ERR_ARG;
    std::vector<SacChanDev> tab(n_ch);
    for (int k = 0; k < n_ch; ++k) {
        const wpcd_channel &ch = channels[k];
        if (ch.J < 0 || ch.J > kMaxJ || (ch.s != 0 && ch.s != 1)) return WPCD_ERR_ARG;
        if (ch.coupled && (ch.s != 1 || ch.J < 1 || ch.l != ch.J - 1 || ch.lp != ch.J + 1)) return WPCD_ERR_ARG;
        if (!ch.coupled && ch.l != ch.lp) return WPCD_ERR_ARG;
        SacChanDev &d = tab[k];
        memset(&d, 0, sizeof(d));
        d.s = ch.s;
        d.J = ch.J;
        d.tz = ch.tz;
        d.K = ch.coupled ? 2 : 1;
        d.l[0] = ch.coupled ? ch.J - 1 : ch.l;
        d.l[1] = ch.coupled ? ch.J + 1 : ch.l;
        for (int ip = 0; ip < d.K; ++ip)
            for (int il = 0; il < d.K; ++il)
                for (int mp = -ch.s; mp <= ch.s; ++mp)
                    for (int m = -ch.s; m <= ch.s; ++m) {
                        const int lp = d.l[ip], l = d.l[il];
                        d.tab[((ip * 2 + il) * 3 + mp + 1) * 3 + m + 1] =
                            std::sqrt(4.0 * kPi) * std::sqrt(2.0 * l + 1.0) *
                            cg_racah(lp, m - mp, ch.s, mp, ch.J, m) * cg_racah(l, 0, ch.s, m, ch.J, m);
                    }
    }
    std::lock_guard<std::mutex> lk(c->mu);
    CK(cudaSetDevice(c->device));
    Exec &X = c->main;
    wpcd_status st = ws_reserve(c, X, X.ws_in, sizeof(SacChanDev) * n_ch);
    if (st) return st;
    CK(cudaMemcpyAsync(X.ws_in.p, tab.data(), sizeof(SacChanDev) * n_ch, cudaMemcpyHostToDevice, X.stream));
    Launch L(c, X, WPCD_PHASE_OBSERVABLES);
    CK(launch_saclay(static_cast<SacChanDev *>(X.ws_in.p), n_ch, S, n_E, e_lab, delta, n_theta, theta, abcde, dsig,
                     X.stream));
    CK(cudaStreamSynchronize(X.stream));  // the channel table lives in a reusable workspace
    return WPCD_OK;
}

// ---- MI comparison method (Sec. 2.1, Sec. 6) ---------------------------------------------------
wpcd_status wpcd_mi_prepare(wpcd_ctx *c, const wpcd_channel *channels, int n_ch, int generator_id,
                            const double *gp_host, int n_gp, int n_terms, int n_quad, double c_map_fm, int *mi_id)
{
    const int gen = generator_id;
    if (!c || !channels || n_ch < 1 || !mi_id || n_quad < 4 || n_quad > kMiMaxNQ || !(c_map_fm > 0) || !gp_host)
        return WPCD_ERR_ARG;
    if (gen == WPCD_GEN_YAMAGUCHI && (n_terms != 1 || n_gp < 2)) return WPCD_ERR_ARG;
    if (gen == WPCD_GEN_YUKAWA && (n_terms < 1 || n_terms > kYukTerms + 1 || n_gp < kYukParams)) return WPCD_ERR_ARG;
    if (gen != WPCD_GEN_YAMAGUCHI && gen != WPCD_GEN_YUKAWA) return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    CK(cudaSetDevice(c->device));
    auto m = std::make_unique<MiH>();
    m->n_ch = n_ch;
    m->NQ = n_quad;
    m->n_terms = n_terms;
    m->gen = gen;
    m->cmap = c_map_fm;
    m->n_gp = n_gp;
    const int M = n_quad + 1;
    size_t vlen = 0;
    int maxJ = 0;
    std::vector<int> work[2];
    for (int k = 0; k < n_ch; ++k) {
        const wpcd_channel &ch = channels[k];
        if (ch.J < 0 || ch.J > kMaxJ || (ch.s != 0 && ch.s != 1)) return WPCD_ERR_ARG;
        if (ch.coupled && (ch.s != 1 || ch.J < 1 || ch.l != ch.J - 1 || ch.lp != ch.J + 1)) return WPCD_ERR_ARG;
        if (!ch.coupled && ch.l != ch.lp) return WPCD_ERR_ARG;
        if (gen == WPCD_GEN_YAMAGUCHI && (ch.coupled || ch.l != 0)) return WPCD_ERR_ARG;
        if (gen == WPCD_GEN_YUKAWA && ch.J > 8) return WPCD_ERR_ARG;
        MiChanDev d;
        memset(&d, 0, sizeof(d));
        d.s = ch.s;
        d.J = ch.J;
        d.l = ch.l;
        d.lp = ch.lp;
        d.coupled = ch.coupled ? 1 : 0;
        d.tz = ch.tz;
        d.K = ch.coupled ? 2 : 1;
        d.n = d.K * M;
        d.vg_off = (long long)vlen;
        vlen += (size_t)n_terms * d.n * d.n;
        m->ch.push_back(d);
        work[d.K - 1].push_back(k);
        maxJ = std::max(maxJ, ch.J);
    }
    m->Lmax = maxJ + 2;
    wpcd_status st;
    if ((st = dalloc(c, &m->ch_dev, (size_t)n_ch)) || (st = dalloc(c, &m->kg, (size_t)n_quad)) ||
        (st = dalloc(c, &m->wg, (size_t)n_quad)) || (st = dalloc(c, &m->gp, (size_t)n_gp)) ||
        (st = dalloc(c, &m->Vg, vlen))) {
        free_mi(c, *m);
        return st;
    }
    for (int K = 0; K < 2; ++K) {
        m->n_work[K] = (int)work[K].size();
        if (work[K].empty()) continue;
        if ((st = dalloc(c, &m->work_dev[K], work[K].size()))) {
            free_mi(c, *m);
            return st;
        }
        CK(cudaMemcpyAsync(m->work_dev[K], work[K].data(), sizeof(int) * work[K].size(), cudaMemcpyHostToDevice,
                           c->main.stream));
    }
    CK(cudaMemcpyAsync(m->ch_dev, m->ch.data(), sizeof(MiChanDev) * n_ch, cudaMemcpyHostToDevice, c->main.stream));
    CK(cudaMemcpyAsync(m->gp, gp_host, sizeof(double) * n_gp, cudaMemcpyHostToDevice, c->main.stream));
    double *glx, *glw, *angx = nullptr, *angw = nullptr;
    if ((st = gl_rule(c, n_quad, &glx, &glw))) return st;
    if (gen == WPCD_GEN_YUKAWA && (st = gl_rule(c, kAngleQ, &angx, &angw))) return st;
    {
        Launch L(c, c->main, WPCD_PHASE_MI);
        CK(launch_mi_grid(n_quad, c_map_fm, glx, glw, m->kg, m->wg, c->main.stream));
    }
    {
        Launch L(c, c->main, WPCD_PHASE_MI);
        CK(launch_mi_pot(gen, m->ch_dev, n_ch, n_quad, m->kg, m->Lmax, m->gp, angx, angw, n_terms, m->Vg,
                         c->main.stream));
    }
    CK(cudaStreamSynchronize(c->main.stream));
    const int id = c->next_id++;
    Handle h;
    h.kind = kMi;
    h.mi = std::move(m);
    c->handles.emplace(id, std::move(h));
    *mi_id = id;
    return WPCD_OK;
}

wpcd_status wpcd_mi_solve(wpcd_ctx *c, int mi_id, const double *coeffs, int S, const double *e_int, int n_I,
                          const double *e_lab, int n_E, double *k_out, double *delta, double *sigma, int *status_dev)
{
    if (!c || S < 1 || !e_int || n_I < 2 || !e_lab || n_E < 1 || (!k_out && !delta && !sigma)) return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    Handle *h = find(c, mi_id, kMi);
    if (!h) return WPCD_ERR_HANDLE;
    MiH &m = *h->mi;
    if (m.n_terms > 1 && !coeffs) return WPCD_ERR_ARG;
    CK(cudaSetDevice(c->device));
    if (!c->n_sm) cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);
    Exec &X = c->main;
    const int M = m.NQ + 1;
    // on-shell columns [ch][n_I][n_terms][K][K][M], phases [S][ch][n_I][3], status [S][ch]
    size_t von_len = 0;
    for (auto &d : m.ch) {
        d.von_off = (long long)von_len;
        von_len += (size_t)n_I * m.n_terms * d.K * d.K * M;
    }
    wpcd_status st;
    const size_t ph_len = (size_t)S * m.n_ch * n_I * 3;
    if ((st = ws_reserve(c, X, X.ws_tbin, (von_len + ph_len) * sizeof(double)))) return st;
    if ((st = ws_reserve(c, X, X.ws_plan_i, (size_t)S * m.n_ch * sizeof(int)))) return st;
    double *Von = static_cast<double *>(X.ws_tbin.p), *ph = Von + von_len;
    int *status = status_dev ? status_dev : static_cast<int *>(X.ws_plan_i.p);
    CK(cudaMemcpyAsync(m.ch_dev, m.ch.data(), sizeof(MiChanDev) * m.n_ch, cudaMemcpyHostToDevice, X.stream));
    double *angx = nullptr, *angw = nullptr;
    if (m.gen == WPCD_GEN_YUKAWA && (st = gl_rule(c, kAngleQ, &angx, &angw))) return st;
    {
        Launch L(c, X, WPCD_PHASE_MI);
        CK(launch_mi_onshell(m.gen, m.ch_dev, m.n_ch, m.NQ, m.kg, n_I, e_int, m.Lmax, m.gp, angx, angw, m.n_terms, Von,
                             X.stream));
    }
    const double *cf = m.n_terms > 1 ? coeffs : nullptr;
    for (int K = 1; K <= 2; ++K) {
        const int nw = m.n_work[K - 1];
        if (!nw) continue;
        const int n = K * M;
        const int per_sm = mi_slots_per_sm(n, m.NQ);
        if (per_sm < 1) return WPCD_ERR_ARG;
        const int items = S * nw;
        const int slots = std::max(1, std::min(items, per_sm * c->n_sm));
        // two FP64 n x n matrices per slot: V, and the rarely used FP64 elimination fallback
        if ((st = ws_reserve(c, X, X.ws_ref, (size_t)slots * 2 * n * n * sizeof(double)))) return st;
        Launch L(c, X, WPCD_PHASE_MI);
        CK(launch_mi_solve(m.ch_dev, m.work_dev[K - 1], nw, n, m.n_ch, S, m.NQ, m.kg, m.wg, m.n_terms, cf, m.Vg, Von,
                           n_I, e_int, static_cast<double *>(X.ws_ref.p), slots, ph, k_out, status, X.err, X.stream));
    }
    if (delta || sigma) {
        Launch L(c, X, WPCD_PHASE_MI);
        CK(launch_mi_observables(m.ch_dev, m.n_ch, S, n_I, e_int, ph, n_E, e_lab, delta, sigma, X.stream));
    }
    return WPCD_OK;
}

}  // extern "C"

// ============================================================================================ serving
//
// Continuous batching.  Requests (one parameter sample, its own energy list,
// an N_WP among the served ones) enter a FIFO queue.  A worker thread owns
// n_slots executors, each with its own CUDA stream and workspaces.  Whenever a
// slot is free and requests wait, the worker takes the oldest request and
// every other queued request with the same (N_WP, precision), up to
// max_batch, and queues one batch on that slot's stream: inputs H2D, the
// eigensolve of every (sample, channel), per-sample energy plans, T, phases and
// cross sections, outputs D2H, and a host callback that marks the slot done.
// Batches on different slots overlap on the device; new requests join the next
// free slot while others run.  Results belong to the context until
// wpcd_release_result.
namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t ticket = 0;
    int model = 0, prec = 0, n_E = 0;
    std::vector<double> coeffs, e_lab;
    Clock::time_point t_submit;
    int state = 0;  // 0 queued, 1 running, 2 done
    wpcd_status status = WPCD_OK;
    std::vector<double> T, delta, sigma;
    double latency_us = 0.0;
    size_t bytes = 0;
};

struct Slot {
    Exec X;
    std::vector<std::shared_ptr<Req>> reqs;
    std::atomic<int> done{0};
    bool busy = false;
    double *pin_in = nullptr, *pin_out = nullptr;
    size_t pin_in_n = 0, pin_out_n = 0;
    int S = 0, nE = 0;
    size_t nt = 0, nd = 0, ns = 0;
};

struct ModelS {
    int n_wp = 0, vset_id = -1;
    std::vector<int> mesh_ids;
    VSetH *v = nullptr;
    double k_top = 0.0;  // kb[N] of its mesh: energies must have p(E) below it
};

}  // namespace

struct Server {
    wpcd_ctx *c = nullptr;
    std::vector<ModelS> models;
    int n_ch = 0, n_terms = 0, max_batch = 64;
    size_t max_queue = 1 << 16;
    std::vector<std::unique_ptr<Slot>> slots;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Req>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<Req>> table;
    uint64_t next_ticket = 1;
    size_t queued_bytes = 0;
    std::thread worker;
    bool stop = false;
    uint64_t completed = 0, batches = 0, batched_requests = 0;
};

namespace {

void CUDART_CB slot_done_cb(void *arg)
{
    Slot *sl = static_cast<Slot *>(arg);
    sl->done.store(1);
}

size_t request_bytes(const ModelS &m, int prec)
{
    size_t b = 0;
    for (const ChanDev &d : m.v->cd) b += (size_t)d.n * d.n * 8 * (prec == WPCD_PREC_MIXED ? 6 : 1) + (size_t)d.n * 8;
    return b + (size_t)m.v->n_ch * m.v->maxN * 11 * 8;
}

// Queue one batch on a slot.  Returns a status for every request of the batch.
wpcd_status launch_batch(Server *sv, Slot &sl)
{
    wpcd_ctx *c = sv->c;
    Exec &X = sl.X;
    const Req &r0 = *sl.reqs[0];
    ModelS &m = sv->models[r0.model];
    VSetH &v = *m.v;
    const int S = (int)sl.reqs.size(), nt1 = std::max(v.n_terms - 1, 1);
    int nE = 0;
    for (auto &r : sl.reqs) nE = std::max(nE, r->n_E);
    sl.S = S;
    sl.nE = nE;
    const size_t in_d = (size_t)S * nt1 + (size_t)S * nE;
    const size_t in_bytes = in_d * 8 + (size_t)S * 4;
    sl.nt = (size_t)S * v.n_ch * nE * 8;
    sl.nd = (size_t)S * v.n_ch * nE * 3;
    sl.ns = (size_t)S * nE;
    // outputs, the slot's device status word, then the per-solve eigensolver status [S][n_ch]
    const size_t out_bytes = (sl.nt + sl.nd + sl.ns) * 8 + 8 + (size_t)S * v.n_ch * 4;
    wpcd_status st;
    if ((st = ws_reserve(c, X, X.ws_in, in_bytes)) || (st = ws_reserve(c, X, X.ws_out, out_bytes))) return st;
    if (sl.pin_in_n < in_bytes) {
        if (sl.pin_in) cudaFreeHost(sl.pin_in);
        sl.pin_in = nullptr;
        CK(cudaMallocHost(&sl.pin_in, in_bytes));
        sl.pin_in_n = in_bytes;
    }
    if (sl.pin_out_n < out_bytes) {
        if (sl.pin_out) cudaFreeHost(sl.pin_out);
        sl.pin_out = nullptr;
        CK(cudaMallocHost(&sl.pin_out, out_bytes));
        sl.pin_out_n = out_bytes;
    }
    double *hc = sl.pin_in, *he = hc + (size_t)S * nt1;
    int *hn = reinterpret_cast<int *>(he + (size_t)S * nE);
    for (int k = 0; k < S; ++k) {
        const Req &r = *sl.reqs[k];
        for (int a = 0; a < nt1; ++a) hc[(size_t)k * nt1 + a] = (a < (int)r.coeffs.size()) ? r.coeffs[a] : 0.0;
        for (int e = 0; e < nE; ++e) he[(size_t)k * nE + e] = r.e_lab[std::min(e, r.n_E - 1)];
        hn[k] = r.n_E;
    }
    double *dc = static_cast<double *>(X.ws_in.p), *de = dc + (size_t)S * nt1;
    int *dn = reinterpret_cast<int *>(de + (size_t)S * nE);
    double *dout = static_cast<double *>(X.ws_out.p);
    CK(cudaMemcpyAsync(dc, hc, in_bytes, cudaMemcpyHostToDevice, X.stream));
    if ((st = run_diag(c, X, v, m.vset_id, v.n_terms > 1 ? dc : nullptr, S, r0.prec, X.eig))) return st;
    PlanDev plan{};
    if ((st = run_tbin(c, X, v, X.eig, de, nE, dn, plan))) return st;
    if ((st = run_outputs(c, X, v, X.eig, nE, plan, dout, dout + sl.nt, dout + sl.nt + sl.nd))) return st;
    CK(cudaMemcpyAsync(dout + sl.nt + sl.nd + sl.ns, X.err, sizeof(int), cudaMemcpyDeviceToDevice, X.stream));
    CK(cudaMemcpyAsync(dout + sl.nt + sl.nd + sl.ns + 1, X.eig.status, sizeof(int) * S * v.n_ch,
                       cudaMemcpyDeviceToDevice, X.stream));
    CK(cudaMemsetAsync(X.err, 0, sizeof(int), X.stream));
    CK(cudaMemcpyAsync(sl.pin_out, dout, out_bytes, cudaMemcpyDeviceToHost, X.stream));
    sl.done.store(0);
    CK(cudaLaunchHostFunc(X.stream, slot_done_cb, &sl));
    return WPCD_OK;
}

void finish_batch(Server *sv, Slot &sl)
{
    const int S = sl.S, nE = sl.nE;
    const ModelS &m = sv->models[sl.reqs[0]->model];
    const int nch = m.v->n_ch;
    const double *T = sl.pin_out, *D = T + sl.nt, *G = D + sl.nd;
    const int derr = *reinterpret_cast<const int *>(G + sl.ns);
    const int *eig_st = reinterpret_cast<const int *>(G + sl.ns + 1);  // [S][n_ch], < 0: not converged
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lk(sv->mu);
    for (int k = 0; k < S; ++k) {
        Req &r = *sl.reqs[k];
        r.T.resize((size_t)nch * r.n_E * 8);
        r.delta.resize((size_t)nch * r.n_E * 3);
        r.sigma.resize(r.n_E);
        for (int ch = 0; ch < nch; ++ch) {
            memcpy(&r.T[(size_t)ch * r.n_E * 8], T + (((size_t)k * nch + ch) * nE) * 8, sizeof(double) * 8 * r.n_E);
            memcpy(&r.delta[(size_t)ch * r.n_E * 3], D + (((size_t)k * nch + ch) * nE) * 3,
                   sizeof(double) * 3 * r.n_E);
        }
        memcpy(r.sigma.data(), G + (size_t)k * nE, sizeof(double) * r.n_E);
        // each request's own status: its solves' convergence; the slot's error word
        // only for errors that are not a property of one sample (energies outside
        // the mesh are refused at submission and never reach a batch)
        bool conv = true;
        for (int ch = 0; ch < nch; ++ch) conv &= eig_st[(size_t)k * nch + ch] >= 0;
        if (!conv) r.status = WPCD_ERR_NOCONVERGE;
        else if (derr == 0 || derr == kDevNoConverge) r.status = WPCD_OK;
        else r.status = derr == kDevTimeout ? WPCD_ERR_TIMEOUT : (derr == kDevBadSize ? WPCD_ERR_CUDA : WPCD_ERR_ARG);
        r.latency_us = std::chrono::duration<double, std::micro>(now - r.t_submit).count();
        r.state = 2;
        sv->queued_bytes -= r.bytes;
    }
    sv->completed += S;
    sl.reqs.clear();
    sl.busy = false;
    sv->cv.notify_all();
}

void fail_batch(Server *sv, Slot &sl, wpcd_status st)
{
    std::lock_guard<std::mutex> lk(sv->mu);
    for (auto &r : sl.reqs) {
        r->status = st;
        r->state = 2;
        sv->queued_bytes -= r->bytes;
    }
    sl.reqs.clear();
    sl.busy = false;
    sv->cv.notify_all();
}

void serve_loop(Server *sv)
{
    cudaSetDevice(sv->c->device);
    for (;;) {
        bool any_busy = false;
        for (auto &slp : sv->slots) {
            Slot &sl = *slp;
            if (sl.busy && sl.done.load()) finish_batch(sv, sl);
            any_busy |= sl.busy;
        }
        for (auto &slp : sv->slots) {
            Slot &sl = *slp;
            if (sl.busy) continue;
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                if (sv->queue.empty()) break;
                const int model = sv->queue.front()->model, prec = sv->queue.front()->prec;
                for (auto it = sv->queue.begin(); it != sv->queue.end() && (int)sl.reqs.size() < sv->max_batch;) {
                    if ((*it)->model == model && (*it)->prec == prec) {
                        (*it)->state = 1;
                        sl.reqs.push_back(*it);
                        it = sv->queue.erase(it);
                    } else {
                        ++it;
                    }
                }
                sv->batches += 1;
                sv->batched_requests += sl.reqs.size();
            }
            sl.busy = true;
            any_busy = true;
            wpcd_status st = launch_batch(sv, sl);
            if (st) {
                cudaStreamSynchronize(sl.X.stream);
                fail_batch(sv, sl, st);
            }
        }
        std::unique_lock<std::mutex> lk(sv->mu);
        if (sv->stop && sv->queue.empty() && !any_busy) break;
        if (sv->queue.empty() || !any_busy)
            sv->cv.wait_for(lk, std::chrono::microseconds(any_busy ? 20 : 2000));
    }
}

}  // namespace

bool serve_owns(wpcd_ctx *c, int id)
{
    if (!c || !c->server) return false;
    for (auto &m : c->server->models) {
        if (m.vset_id == id) return true;
        for (int mid : m.mesh_ids)
            if (mid == id) return true;
    }
    return false;
}

void serve_shutdown(wpcd_ctx *c)
{
    Server *sv = c->server;
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    for (auto &slp : sv->slots) {
        Slot &sl = *slp;
        cudaStreamSynchronize(sl.X.stream);
        free_eig(c, sl.X.eig);
        for (auto *b : {&sl.X.ws_plan_i, &sl.X.ws_plan_d, &sl.X.ws_tbin, &sl.X.ws_phbin, &sl.X.ws_ref, &sl.X.ws_in,
                        &sl.X.ws_out})
            dfree(c, b->p);
        dfree(c, sl.X.err);
        if (sl.pin_in) cudaFreeHost(sl.pin_in);
        if (sl.pin_out) cudaFreeHost(sl.pin_out);
        cudaStreamDestroy(sl.X.stream);
    }
    c->server = nullptr;
    delete sv;
}

extern "C" {

wpcd_status wpcd_serve_start(wpcd_ctx *c, const wpcd_channel *channels, int n_ch, int generator_id,
                             const double *gen_params_host, int n_gen_params, int n_terms, const int *n_wp_list,
                             int n_nwp, int max_batch, int n_slots, int max_queue)
{
    if (!c || !channels || n_ch < 1 || !n_wp_list || n_nwp < 1 || max_batch < 1 || n_slots < 1 || n_slots > 16 ||
        max_queue < 1 || generator_id == WPCD_GEN_FINE)
        return WPCD_ERR_ARG;
    if (c->server) return WPCD_ERR_ARG;
    auto sv = std::make_unique<Server>();
    sv->c = c;
    sv->n_ch = n_ch;
    sv->n_terms = n_terms;
    sv->max_batch = max_batch;
    sv->max_queue = (size_t)max_queue;
    wpcd_status st;
    for (int k = 0; k < n_nwp; ++k) {
        ModelS m;
        m.n_wp = n_wp_list[k];
        int mid = -1;
        if ((st = wpcd_mesh(c, m.n_wp, 0, 100.0 / kHbarc, 2.0, 8.0, 8, 0, &mid))) return st;
        m.mesh_ids.assign(n_ch, mid);
        if ((st = wpcd_project(c, m.mesh_ids.data(), channels, n_ch, generator_id, gen_params_host, n_gen_params,
                               nullptr, n_terms, &m.vset_id)))
            return st;
        {
            std::lock_guard<std::mutex> lk(c->mu);
            m.v = find(c, m.vset_id, kVSet)->vset.get();
            const MeshH &mh = *find(c, mid, kMesh)->mesh;
            CK(cudaMemcpy(&m.k_top, mh.kb + mh.N, sizeof(double), cudaMemcpyDeviceToHost));
        }
        sv->models.push_back(m);
    }
    CK(cudaSetDevice(c->device));
    for (int k = 0; k < n_slots; ++k) {
        auto sl = std::make_unique<Slot>();
        CK(cudaStreamCreateWithFlags(&sl->X.stream, cudaStreamNonBlocking));
        if ((st = dalloc(c, &sl->X.err, 1))) return st;
        CK(cudaMemsetAsync(sl->X.err, 0, sizeof(int), sl->X.stream));
        sv->slots.push_back(std::move(sl));
    }
    CK(cudaStreamSynchronize(c->main.stream));
    Server *raw = sv.release();
    c->server = raw;
    raw->worker = std::thread(serve_loop, raw);
    return WPCD_OK;
}

wpcd_status wpcd_serve_stop(wpcd_ctx *c)
{
    if (!c || !c->server) return WPCD_ERR_ARG;
    serve_shutdown(c);
    return WPCD_OK;
}

wpcd_status wpcd_submit(wpcd_ctx *c, const wpcd_request *rq, uint64_t *ticket)
{
    if (!c || !c->server || !rq || !ticket || !rq->e_lab || rq->n_E < 1) return WPCD_ERR_ARG;
    Server *sv = c->server;
    if (rq->prec != WPCD_PREC_FP64 && rq->prec != WPCD_PREC_MIXED) return WPCD_ERR_ARG;
    if (sv->n_terms > 1 && (!rq->coeffs || rq->n_terms != sv->n_terms - 1)) return WPCD_ERR_ARG;
    int model = -1;
    for (size_t k = 0; k < sv->models.size(); ++k)
        if (sv->models[k].n_wp == rq->n_wp) model = (int)k;
    if (model < 0) return WPCD_ERR_ARG;
    if (sv->models[model].v->maxn > jacobi_big_max_n()) return WPCD_ERR_ARG;
    // the energy plan's test, on the host: a request with an energy outside the
    // mesh is refused here instead of failing the batch it would join
    for (int e = 0; e < rq->n_E; ++e) {
        const double T = rq->e_lab[e];
        if (!(T > 0.0) || !(std::sqrt(kMn * T / 2.0) / kHbarc < sv->models[model].k_top)) return WPCD_ERR_ARG;
    }
    auto r = std::make_shared<Req>();
    r->model = model;
    r->prec = rq->prec;
    r->n_E = rq->n_E;
    if (sv->n_terms > 1) r->coeffs.assign(rq->coeffs, rq->coeffs + rq->n_terms);
    r->e_lab.assign(rq->e_lab, rq->e_lab + rq->n_E);
    r->bytes = request_bytes(sv->models[model], rq->prec);
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return WPCD_ERR_ARG;
    const size_t cap = c->budget ? (c->budget > c->in_use ? c->budget - c->in_use : 0) : (size_t)-1;
    if (sv->queue.size() >= sv->max_queue || (c->budget && sv->queued_bytes + r->bytes > cap))
        return WPCD_ERR_BUDGET;
    r->ticket = sv->next_ticket++;
    r->t_submit = Clock::now();
    sv->queued_bytes += r->bytes;
    sv->queue.push_back(r);
    sv->table[r->ticket] = r;
    *ticket = r->ticket;
    sv->cv.notify_all();
    return WPCD_OK;
}

static void fill_result(const Req &r, int n_ch, wpcd_result *out)
{
    out->status = r.status;
    out->n_E = r.n_E;
    out->n_ch = n_ch;
    out->delta = r.delta.data();
    out->sigma = r.sigma.data();
    out->T = r.T.data();
    out->latency_us = r.latency_us;
}

wpcd_status wpcd_poll(wpcd_ctx *c, uint64_t ticket, wpcd_result *out)
{
    if (!c || !c->server || !out) return WPCD_ERR_ARG;
    Server *sv = c->server;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->table.find(ticket);
    if (it == sv->table.end()) return WPCD_ERR_HANDLE;
    if (it->second->state != 2) return WPCD_ERR_NOTREADY;
    fill_result(*it->second, sv->n_ch, out);
    return WPCD_OK;
}

wpcd_status wpcd_wait(wpcd_ctx *c, uint64_t ticket, int timeout_ms, wpcd_result *out)
{
    if (!c || !c->server || !out) return WPCD_ERR_ARG;
    Server *sv = c->server;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->table.find(ticket);
    if (it == sv->table.end()) return WPCD_ERR_HANDLE;
    std::shared_ptr<Req> r = it->second;
    if (!sv->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->state == 2; }))
        return WPCD_ERR_TIMEOUT;
    fill_result(*r, sv->n_ch, out);
    return WPCD_OK;
}

void wpcd_release_result(wpcd_ctx *c, uint64_t ticket)
{
    if (!c || !c->server) return;
    std::lock_guard<std::mutex> lk(c->server->mu);
    auto it = c->server->table.find(ticket);
    if (it != c->server->table.end() && it->second->state == 2) c->server->table.erase(it);
}

wpcd_status wpcd_serve_stats(wpcd_ctx *c, unsigned long long *completed, unsigned long long *batches,
                             unsigned long long *queued)
{
    if (!c || !c->server) return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->server->mu);
    if (completed) *completed = c->server->completed;
    if (batches) *batches = c->server->batches;
    if (queued) *queued = c->server->queue.size();
    return WPCD_OK;
}

}  // extern "C"
