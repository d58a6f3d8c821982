// runtime.cu -- host runtime of libwpcd: context, handle tables, device-memory
// accounting against the HBM budget, size buckets, and the C ABI of wpcd.h.
// Every numerical step runs in the kernels of the other translation units;
// this file only allocates, validates, orders launches and copies.
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "wpcd_internal.cuh"

namespace wpcd {
size_t tbin_smem_bytes(int nmax);
}

using namespace wpcd;

namespace {

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
};

struct EigH {
    int vset_id = -1, n_samples = 0;
    double *eps = nullptr, *C = nullptr, *coeffs = nullptr;
    int *status = nullptr;
    ChanDev *cd_dev = nullptr;  // vset channels with this eig's offsets
    size_t eps_len = 0, c_len = 0, coeff_len = 0;
};

enum Kind { kMesh = 1, kVSet = 2, kEig = 3 };

struct Handle {
    Kind kind;
    std::unique_ptr<MeshH> mesh;
    std::unique_ptr<VSetH> vset;
    std::unique_ptr<EigH> eig;
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
    int *err_dev = nullptr;
    // Gauss-Legendre rules cached on the device, keyed by order
    std::map<int, std::pair<double *, double *>> gl;
    // grow-only workspaces
    struct Buf {
        void *p = nullptr;
        size_t n = 0;
    };
    Buf ws_plan_i, ws_plan_d, ws_tbin, ws_phbin, ws_in, ws_out;
    void *pin_in = nullptr, *pin_out = nullptr;
    size_t pin_in_n = 0, pin_out_n = 0;
    EigH scratch_eig;  // eigenpairs of wpcd_solve
    // tracing: kernels launched, and (when enabled) CUDA events around each launch
    unsigned long long launches = 0;
    bool prof = false;
    struct Rec {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    double prof_ms[WPCD_PHASE_COUNT] = {};
    long prof_n[WPCD_PHASE_COUNT] = {};
};

namespace {

#define CK(call)                                      \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return WPCD_ERR_CUDA; \
    } while (0)

wpcd_status dmalloc(wpcd_ctx *c, void **p, size_t bytes)
{
    if (bytes == 0) bytes = 8;
    if (c->budget && c->in_use + bytes > c->budget) return WPCD_ERR_BUDGET;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return WPCD_ERR_NOMEM;
    }
    c->in_use += bytes;
    c->sizes[*p] = bytes;
    return WPCD_OK;
}

void dfree(wpcd_ctx *c, void *p)
{
    if (!p) return;
    auto it = c->sizes.find(p);
    if (it != c->sizes.end()) {
        c->in_use -= it->second;
        c->sizes.erase(it);
    }
    cudaFree(p);
}

template <class T>
wpcd_status dalloc(wpcd_ctx *c, T **p, size_t count)
{
    return dmalloc(c, reinterpret_cast<void **>(p), count * sizeof(T));
}

// Counts one kernel launch of `phase`; with profiling on, brackets it with events.
struct Launch {
    wpcd_ctx *c;
    wpcd_ctx::Rec r{};
    Launch(wpcd_ctx *cc, int phase) : c(cc)
    {
        ++c->launches;
        r.phase = phase;
        if (c->prof) {
            cudaEventCreate(&r.a);
            cudaEventCreate(&r.b);
            cudaEventRecord(r.a, c->stream);
        }
    }
    ~Launch()
    {
        if (c->prof) {
            cudaEventRecord(r.b, c->stream);
            c->recs.push_back(r);
        }
    }
};

void prof_collect(wpcd_ctx *c)
{
    if (c->recs.empty()) return;
    cudaStreamSynchronize(c->stream);
    for (auto &r : c->recs) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        c->prof_ms[r.phase] += ms;
        c->prof_n[r.phase] += 1;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    c->recs.clear();
}

wpcd_status ws_reserve(wpcd_ctx *c, wpcd_ctx::Buf &b, size_t bytes)
{
    if (b.n >= bytes) return WPCD_OK;
    if (b.p) {
        cudaStreamSynchronize(c->stream);
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
        Launch L(c, WPCD_PHASE_MESH);
        CK(launch_gauss_legendre(n, dx, dw, c->stream));
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
    e = EigH();
}

void free_vset(wpcd_ctx *c, VSetH &v)
{
    dfree(c, v.V);
    dfree(c, v.cd_dev);
    dfree(c, v.ident_dev);
    for (auto &kv : v.bucket_dev) dfree(c, kv.second);
}

void free_mesh(wpcd_ctx *c, MeshH &m)
{
    dfree(c, m.kb);
    dfree(c, m.kq);
    dfree(c, m.wq);
    dfree(c, m.h0);
}

// Allocate (or reuse) eigenpair storage for `S` samples of vset v and run the
// parameter sum + eigensolve.
wpcd_status run_diag(wpcd_ctx *c, VSetH &v, int vset_id, const double *coeffs, int S, EigH &e)
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
    if (e.eps_len < eps_len || e.c_len < c_len || e.coeff_len < coeff_len || e.n_samples != S ||
        e.vset_id != vset_id || !e.cd_dev) {
        cudaStreamSynchronize(c->stream);
        free_eig(c, e);
        if ((st = dalloc(c, &e.eps, eps_len))) return st;
        if ((st = dalloc(c, &e.C, c_len))) return st;
        if ((st = dalloc(c, &e.coeffs, coeff_len))) return st;
        if ((st = dalloc(c, &e.status, (size_t)S * v.n_ch))) return st;
        if ((st = dalloc(c, &e.cd_dev, (size_t)v.n_ch))) return st;
        e.eps_len = eps_len;
        e.c_len = c_len;
        e.coeff_len = coeff_len;
    }
    e.vset_id = vset_id;
    e.n_samples = S;
    CK(cudaMemcpyAsync(e.cd_dev, cd.data(), sizeof(ChanDev) * v.n_ch, cudaMemcpyHostToDevice, c->stream));
    if (v.n_terms > 1) {
        CK(cudaMemcpyAsync(e.coeffs, coeffs, sizeof(double) * S * (v.n_terms - 1), cudaMemcpyDeviceToDevice,
                           c->stream));
    }
    const double *cf = v.n_terms > 1 ? e.coeffs : nullptr;
    if (c->exec_mode == WPCD_EXEC_PLAIN) {
        // one solve per launch: the baseline execution on the same GPU
        for (int s = 0; s < S; ++s)
            for (int k = 0; k < v.n_ch; ++k)
                CK((Launch(c, WPCD_PHASE_EIGEN), launch_jacobi_f64(e.cd_dev, v.ident_dev + k, 1, 1, s, v.n_terms, cf, cd[k].n, e.eps, e.C, e.status,
                                     v.n_ch, c->err_dev, c->stream)));
    } else {
        // one launch per size bucket, largest first
        for (auto it = v.buckets.rbegin(); it != v.buckets.rend(); ++it) {
            const int n = it->first;
            const int nw = (int)it->second.size();
            Launch L(c, WPCD_PHASE_EIGEN);
            CK(launch_jacobi_f64(e.cd_dev, v.bucket_dev[n], nw, S, 0, v.n_terms, cf, n, e.eps, e.C, e.status, v.n_ch,
                                 c->err_dev, c->stream));
        }
    }
    return WPCD_OK;
}

// Energy plan + T at the needed bins into the context workspaces.
wpcd_status run_tbin(wpcd_ctx *c, VSetH &v, EigH &e, const double *e_lab, int n_E, PlanDev &plan)
{
    const int nch = v.n_ch, maxN = v.maxN, S = e.n_samples;
    wpcd_status st;
    const size_t ni = (size_t)2 * nch * n_E + nch + (size_t)nch * maxN;
    if ((st = ws_reserve(c, c->ws_plan_i, ni * sizeof(int)))) return st;
    if ((st = ws_reserve(c, c->ws_plan_d, (size_t)n_E * sizeof(double)))) return st;
    if ((st = ws_reserve(c, c->ws_tbin, (size_t)S * nch * maxN * 8 * sizeof(double)))) return st;
    if ((st = ws_reserve(c, c->ws_phbin, (size_t)S * nch * maxN * 3 * sizeof(double)))) return st;
    int *pi = static_cast<int *>(c->ws_plan_i.p);
    plan.bin = pi;
    plan.brk = pi + (size_t)nch * n_E;
    plan.cnt = plan.brk + (size_t)nch * n_E;
    plan.list = plan.cnt + nch;
    plan.pE = static_cast<double *>(c->ws_plan_d.p);
    {
        Launch L(c, WPCD_PHASE_PLAN);
        CK(launch_plan(e.cd_dev, nch, maxN, e_lab, n_E, plan, c->err_dev, c->stream));
    }
    Launch L(c, WPCD_PHASE_TMATRIX);
    CK(launch_tbin(e.cd_dev, nch, S, v.n_terms, v.n_terms > 1 ? e.coeffs : nullptr, e.eps, e.C, plan, maxN,
                   static_cast<double *>(c->ws_tbin.p), static_cast<double *>(c->ws_phbin.p), c->err_dev, c->stream));
    return WPCD_OK;
}

wpcd_status check_energies(const double *e_lab, int n_E)
{
    if (!e_lab || n_E < 1) return WPCD_ERR_ARG;
    return WPCD_OK;
}

}  // namespace

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
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->budget = hbm_budget_bytes;
    if (dalloc(c, &c->err_dev, 1) != WPCD_OK || cudaMemsetAsync(c->err_dev, 0, sizeof(int), c->stream) != cudaSuccess) {
        delete c;
        return WPCD_ERR_CUDA;
    }
    *out = c;
    return WPCD_OK;
}

void wpcd_destroy(wpcd_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (auto &kv : c->handles) {
        if (kv.second.mesh) free_mesh(c, *kv.second.mesh);
        if (kv.second.vset) free_vset(c, *kv.second.vset);
        if (kv.second.eig) free_eig(c, *kv.second.eig);
    }
    free_eig(c, c->scratch_eig);
    for (auto &kv : c->gl) {
        dfree(c, kv.second.first);
        dfree(c, kv.second.second);
    }
    for (auto *b : {&c->ws_plan_i, &c->ws_plan_d, &c->ws_tbin, &c->ws_phbin, &c->ws_in, &c->ws_out}) dfree(c, b->p);
    if (c->pin_in) cudaFreeHost(c->pin_in);
    if (c->pin_out) cudaFreeHost(c->pin_out);
    dfree(c, c->err_dev);
    delete c;
}

wpcd_status wpcd_set_option(wpcd_ctx *c, int key, int value)
{
    if (!c) return WPCD_ERR_ARG;
    if (key == WPCD_OPT_EXEC && (value == WPCD_EXEC_BATCHED || value == WPCD_EXEC_PLAIN)) {
        c->exec_mode = value;
        return WPCD_OK;
    }
    return WPCD_ERR_ARG;
}

wpcd_status wpcd_sync(wpcd_ctx *c)
{
    if (!c) return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    CK(cudaSetDevice(c->device));
    int h = 0;
    CK(cudaMemcpyAsync(&h, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (h != 0) CK(cudaMemsetAsync(c->err_dev, 0, sizeof(int), c->stream));
    switch (h) {
    case kDevOk: return WPCD_OK;
    case kDevEnergyOutside: return WPCD_ERR_ARG;
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
    Launch L(c, WPCD_PHASE_MESH);
    CK(launch_mesh(n_wp, kind, alpha, t, kmax, n_quad, wp_kind, glx, glw, m->kb, m->kq, m->wq, m->h0, c->stream));
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
    if (kb) CK(cudaMemcpyAsync(kb, m.kb, sizeof(double) * (m.N + 1), cudaMemcpyDeviceToHost, c->stream));
    if (kq) CK(cudaMemcpyAsync(kq, m.kq, sizeof(double) * m.N * m.Q, cudaMemcpyDeviceToHost, c->stream));
    if (wq) CK(cudaMemcpyAsync(wq, m.wq, sizeof(double) * m.N * m.Q, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return WPCD_OK;
}

wpcd_status wpcd_project(wpcd_ctx *c, const int *mesh_ids, const wpcd_channel *chs, int n_ch, int gen,
                         const double *gp_host, int n_gp, const double *v_fine_dev, int n_terms, int *vset_id)
{
    if (!c || !mesh_ids || !chs || n_ch < 1 || !vset_id || n_terms < 1 || n_terms > kMaxTerms) return WPCD_ERR_ARG;
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
    CK(cudaMemcpyAsync(v->cd_dev, v->cd.data(), sizeof(ChanDev) * n_ch, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(v->ident_dev, ident.data(), sizeof(int) * n_ch, cudaMemcpyHostToDevice, c->stream));
    for (auto &kv : v->buckets) {
        int *p;
        if ((st = dalloc(c, &p, kv.second.size()))) {
            free_vset(c, *v);
            return st;
        }
        v->bucket_dev[kv.first] = p;
        CK(cudaMemcpyAsync(p, kv.second.data(), sizeof(int) * kv.second.size(), cudaMemcpyHostToDevice, c->stream));
    }
    if (gen == WPCD_GEN_FINE) {
        size_t off = 0;
        for (int k = 0; k < n_ch; ++k) {
            const ChanDev &d = v->cd[k];
            Launch L(c, WPCD_PHASE_PROJECT);
            CK(launch_project_fine(v->cd_dev, k, d, v_fine_dev + off, n_terms, c->stream));
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
        CK(cudaMemcpyAsync(gp_dev, gp_host, sizeof(double) * n_gp, cudaMemcpyHostToDevice, c->stream));
        double *angx = nullptr, *angw = nullptr;
        if (gen == WPCD_GEN_YUKAWA && (st = gl_rule(c, kAngleQ, &angx, &angw))) return st;
        // group the channels by mesh; one launch per mesh
        std::map<int, std::vector<int>> groups;
        for (int k = 0; k < n_ch; ++k) groups[mesh_ids[k]].push_back(k);
        std::vector<int *> gdevs;
        for (auto &kv : groups) {
            int *gd;
            if ((st = dalloc(c, &gd, kv.second.size()))) return st;
            gdevs.push_back(gd);
            CK(cudaMemcpyAsync(gd, kv.second.data(), sizeof(int) * kv.second.size(), cudaMemcpyHostToDevice,
                               c->stream));
            const ChanDev &d0 = v->cd[kv.second[0]];
            Launch L(c, WPCD_PHASE_PROJECT);
            if (gen == WPCD_GEN_YUKAWA)
                CK(launch_project_yukawa(v->cd_dev, gd, (int)kv.second.size(), d0.N, d0.Q, maxJ + 2, gp_dev, angx, angw,
                                         n_terms, c->stream));
            else
                CK(launch_project_yamaguchi_gp(v->cd_dev, gd, (int)kv.second.size(), d0.N, d0.Q, gp_dev, c->stream));
        }
        CK(cudaStreamSynchronize(c->stream));
        for (int *gd : gdevs) dfree(c, gd);
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
    CK(cudaMemcpyAsync(out, d.V, sizeof(double) * v.n_terms * d.n * d.n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return WPCD_OK;
}

wpcd_status wpcd_diag(wpcd_ctx *c, int vset_id, const double *coeffs_dev, int n_samples, wpcd_precision prec,
                      int *eig_id)
{
    if (!c || !eig_id || n_samples < 1 || prec != WPCD_PREC_FP64) return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    Handle *h = find(c, vset_id, kVSet);
    if (!h) return WPCD_ERR_HANDLE;
    VSetH &v = *h->vset;
    if (v.n_terms > 1 && !coeffs_dev) return WPCD_ERR_ARG;
    CK(cudaSetDevice(c->device));
    auto e = std::make_unique<EigH>();
    wpcd_status st = run_diag(c, v, vset_id, coeffs_dev, n_samples, *e);
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
                       c->stream));
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
                           c->stream));
    if (C_host)
        CK(cudaMemcpyAsync(C_host, e.C + co + (size_t)sample * n * n, sizeof(double) * n * n, cudaMemcpyDeviceToHost,
                           c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return WPCD_OK;
}

static wpcd_status tmatrix_impl(wpcd_ctx *c, VSetH &v, EigH &e, const double *e_lab, int n_E, double *t_out,
                                double *delta, double *sigma)
{
    PlanDev plan;
    wpcd_status st = run_tbin(c, v, e, e_lab, n_E, plan);
    if (st) return st;
    if (t_out)
        CK((Launch(c, WPCD_PHASE_GATHER), launch_gather_t(e.cd_dev, v.n_ch, e.n_samples, n_E, v.maxN, plan, static_cast<double *>(c->ws_tbin.p), t_out,
                           c->stream)));
    if (delta || sigma)
        CK((Launch(c, WPCD_PHASE_OBSERVABLES), launch_observables(e.cd_dev, v.n_ch, e.n_samples, n_E, v.maxN, plan, static_cast<double *>(c->ws_phbin.p),
                              delta, sigma, c->stream)));
    return WPCD_OK;
}

wpcd_status wpcd_tmatrix(wpcd_ctx *c, int eig_id, const double *e_lab, int n_E, wpcd_resolvent res, double *t_out)
{
    if (!c || !t_out || res != WPCD_AVG_FREE_BIN || check_energies(e_lab, n_E)) return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    Handle *h = find(c, eig_id, kEig);
    if (!h) return WPCD_ERR_HANDLE;
    Handle *hv = find(c, h->eig->vset_id, kVSet);
    if (!hv) return WPCD_ERR_HANDLE;
    CK(cudaSetDevice(c->device));
    return tmatrix_impl(c, *hv->vset, *h->eig, e_lab, n_E, t_out, nullptr, nullptr);
}

wpcd_status wpcd_observables(wpcd_ctx *c, int eig_id, const double *e_lab, int n_E, double *delta, double *sigma)
{
    if (!c || check_energies(e_lab, n_E) || (!delta && !sigma)) return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    Handle *h = find(c, eig_id, kEig);
    if (!h) return WPCD_ERR_HANDLE;
    Handle *hv = find(c, h->eig->vset_id, kVSet);
    if (!hv) return WPCD_ERR_HANDLE;
    CK(cudaSetDevice(c->device));
    return tmatrix_impl(c, *hv->vset, *h->eig, e_lab, n_E, nullptr, delta, sigma);
}

wpcd_status wpcd_solve(wpcd_ctx *c, int vset_id, const double *coeffs, int S, const double *e_lab, int n_E,
                       wpcd_precision prec, wpcd_resolvent res, double *t_out, double *delta, double *sigma)
{
    if (!c || S < 1 || prec != WPCD_PREC_FP64 || res != WPCD_AVG_FREE_BIN || check_energies(e_lab, n_E))
        return WPCD_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    Handle *hv = find(c, vset_id, kVSet);
    if (!hv) return WPCD_ERR_HANDLE;
    VSetH &v = *hv->vset;
    if (v.n_terms > 1 && !coeffs) return WPCD_ERR_ARG;
    CK(cudaSetDevice(c->device));
    wpcd_status st = run_diag(c, v, vset_id, coeffs, S, c->scratch_eig);
    if (st) return st;
    return tmatrix_impl(c, v, c->scratch_eig, e_lab, n_E, t_out, delta, sigma);
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
    double *din, *dout, *hin, *hout;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        CK(cudaSetDevice(c->device));
        if ((st = ws_reserve(c, c->ws_in, in_bytes)) || (st = ws_reserve(c, c->ws_out, out_bytes))) return st;
        if (c->pin_in_n < in_bytes) {
            if (c->pin_in) cudaFreeHost(c->pin_in);
            CK(cudaMallocHost(&c->pin_in, in_bytes));
            c->pin_in_n = in_bytes;
        }
        if (c->pin_out_n < out_bytes) {
            if (c->pin_out) cudaFreeHost(c->pin_out);
            CK(cudaMallocHost(&c->pin_out, out_bytes));
            c->pin_out_n = out_bytes;
        }
        din = static_cast<double *>(c->ws_in.p);
        dout = static_cast<double *>(c->ws_out.p);
        hin = static_cast<double *>(c->pin_in);
        hout = static_cast<double *>(c->pin_out);
        if (nc) memcpy(hin, coeffs_h, nc * sizeof(double));
        memcpy(hin + nc, e_lab_h, n_E * sizeof(double));
        CK(cudaMemcpyAsync(din, hin, in_bytes, cudaMemcpyHostToDevice, c->stream));
    }
    st = wpcd_solve(c, vset_id, nc ? din : nullptr, S, din + nc, n_E, prec, res, t_h ? dout : nullptr,
                    delta_h ? dout + nt : nullptr, sigma_h ? dout + nt + nd : nullptr);
    if (st) return st;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        if (out_bytes) CK(cudaMemcpyAsync(hout, dout, out_bytes, cudaMemcpyDeviceToHost, c->stream));
    }
    st = wpcd_sync(c);
    if (t_h) memcpy(t_h, hout, nt * sizeof(double));
    if (delta_h) memcpy(delta_h, hout + nt, nd * sizeof(double));
    if (sigma_h) memcpy(sigma_h, hout + nt + nd, ns * sizeof(double));
    return st;
}

unsigned long long wpcd_kernel_launches(const wpcd_ctx *c) { return c ? c->launches : 0; }

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
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->handles.find(id);
    if (it == c->handles.end()) return WPCD_ERR_HANDLE;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (it->second.mesh) free_mesh(c, *it->second.mesh);
    if (it->second.vset) free_vset(c, *it->second.vset);
    if (it->second.eig) free_eig(c, *it->second.eig);
    c->handles.erase(it);
    return WPCD_OK;
}

}  // extern "C"
