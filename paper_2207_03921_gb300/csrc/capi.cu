// C ABI of libnlfem.so (declared in include/nlfem.h): handles, argument checks, the
// assembly driver with its per-mesh cache, and thread-local error messages.
#include <cmath>
#include <cstring>
#include <new>

#include <mutex>
#include <vector>
#include <algorithm>
#include "nlfem_internal.cuh"
#include "rules_table.h"

namespace nlfem {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

static bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T>
static void upload(DBuf<T>& dst, const void* src, size_t count, cudaStream_t st) {
    dst.alloc(count, st);
    if (!count) return;
    cudaMemcpyKind kind = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    NLFEM_CUDA_TRY(cudaMemcpyAsync(dst.p, src, count * sizeof(T), kind, st));
}

static void fill_rule(Rule& r, int n) {
    const double(*tab)[4] = n == 7 ? NLFEM_RULE7 : NLFEM_RULE16;
    r.n = n;
    for (int i = 0; i < n; ++i) {
        r.l[i][0] = tab[i][0];
        r.l[i][1] = tab[i][1];
        r.l[i][2] = tab[i][2];
        r.w[i] = tab[i][3];
    }
}

static void fill_gauss(DuffyRule& d, int n) {
    d.n = n;
    if (n == 5) {
        for (int i = 0; i < 5; ++i) {
            d.x[i] = NLFEM_GAUSS5_X[i];
            d.w[i] = NLFEM_GAUSS5_W[i];
        }
    } else {
        // Gauss-Legendre on (0,1) by Newton iteration on P_n (any n up to 32)
        for (int i = 0; i < n; ++i) {
            double x = std::cos(M_PI * (i + 0.75) / (n + 0.5));
            double dp = 1.0;
            for (int it = 0; it < 100; ++it) {
                double p0 = 1.0, p1 = x;
                for (int k = 2; k <= n; ++k) {
                    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = p2;
                }
                dp = n * (x * p1 - p0) / (x * x - 1.0);
                double dx = p1 / dp;
                x -= dx;
                if (std::fabs(dx) < 1e-17) break;
            }
            d.x[n - 1 - i] = 0.5 * (x + 1.0);
            d.w[n - 1 - i] = 1.0 / ((1.0 - x * x) * dp * dp);
        }
    }
    d.sum_w = 0.0;
    d.sum_wx = 0.0;
    for (int i = 0; i < n; ++i) {
        d.sum_w += d.w[i];
        d.sum_wx += d.w[i] * d.x[i];
    }
}

static Params make_params(const nlfem_params& p, int ndof) {
    NLFEM_CHECK(p.kernel >= 0 && p.kernel <= 3, NLFEM_ERR_INVALID_ARG, "unknown kernel");
    if (p.kernel == NLFEM_KERNEL_TABULATED) {
        NLFEM_CHECK(p.kernel_table && p.table_size >= 2 && p.table_size <= 1024, NLFEM_ERR_INVALID_ARG,
                    "the tabulated kernel needs a table of 2..1024 values");
        for (int i = 0; i < p.table_size; ++i)
            NLFEM_CHECK(std::isfinite(p.kernel_table[i]), NLFEM_ERR_INVALID_ARG, "kernel_table must be finite");
    }
    NLFEM_CHECK(p.delta > 0 && std::isfinite(p.delta), NLFEM_ERR_INVALID_ARG, "delta must be > 0");
    NLFEM_CHECK(p.ball == NLFEM_BALL_NOCAPS || p.ball == NLFEM_BALL_APPROXCAPS || p.ball == NLFEM_BALL_INFINITY,
                NLFEM_ERR_INVALID_ARG, "unknown ball");
    NLFEM_CHECK((p.quad_outer == 7 || p.quad_outer == 16) && (p.quad_inner == 7 || p.quad_inner == 16),
                NLFEM_ERR_INVALID_ARG, "quadrature rules must have 7 or 16 points");
    NLFEM_CHECK(p.close_rule >= 0 && p.close_rule <= 3, NLFEM_ERR_INVALID_ARG, "unknown close-pair rule");
    NLFEM_CHECK(p.precision == NLFEM_PREC_FP64 || p.precision == NLFEM_PREC_FP32_BULK, NLFEM_ERR_INVALID_ARG,
                "unknown precision");
    NLFEM_CHECK(p.n_materials >= 0 && p.n_materials <= 16 && (p.n_materials == 0 || p.material_scale),
                NLFEM_ERR_INVALID_ARG, "n_materials must be 0..16 with a material_scale table");
    for (int a = 0; a < p.n_materials; ++a)
        for (int b = 0; b < p.n_materials; ++b) {
            const double x = p.material_scale[a * p.n_materials + b];
            NLFEM_CHECK(std::isfinite(x) && x == p.material_scale[b * p.n_materials + a], NLFEM_ERR_INVALID_ARG,
                        "material_scale must be finite and symmetric");
        }
    NLFEM_CHECK(p.duffy_gauss >= 1 && p.duffy_gauss <= 32, NLFEM_ERR_INVALID_ARG,
                "duffy_gauss must be in 1..32");
    NLFEM_CHECK(p.singular_precision == NLFEM_SINGULAR_FP64 || p.singular_precision == NLFEM_SINGULAR_FP32,
                NLFEM_ERR_INVALID_ARG, "unknown singular_precision");
    NLFEM_CHECK(p.geometry_precision == NLFEM_GEOMETRY_FP32 || p.geometry_precision == NLFEM_GEOMETRY_FP64,
                NLFEM_ERR_INVALID_ARG, "unknown geometry_precision");
    int need = p.kernel == NLFEM_KERNEL_PERIDYNAMIC ? 2 : 1;
    NLFEM_CHECK(need == ndof, NLFEM_ERR_INVALID_ARG, "the mesh was created with the wrong dofs per node for this kernel");
    if (p.kernel == NLFEM_KERNEL_FRACTIONAL)
        NLFEM_CHECK(p.s > 0.0 && p.s < 1.0, NLFEM_ERR_INVALID_ARG, "fractional kernel needs 0 < s < 1");
    Params P;
    std::memset(&P, 0, sizeof P);
    P.kernel = p.kernel;
    P.ball = p.ball;
    P.close_rule = p.close_rule;
    P.precision = p.precision;
    P.ndof = ndof;
    // the arithmetic switches only apply to FP32 bulk (the FP64 path is FP64 throughout)
    P.sing32 = p.precision == NLFEM_PREC_FP32_BULK && p.singular_precision == NLFEM_SINGULAR_FP32;
    P.geo64 = p.precision == NLFEM_PREC_FP32_BULK && p.geometry_precision == NLFEM_GEOMETRY_FP64;
    P.delta = p.delta;
    P.delta2 = p.delta * p.delta;
    P.s = p.kernel == NLFEM_KERNEL_FRACTIONAL ? p.s : (p.kernel == NLFEM_KERNEL_PERIDYNAMIC ? -0.5 : -1.0);
    if (!std::isnan(p.kconst)) P.c = p.kconst;
    else if (p.kernel == NLFEM_KERNEL_CONSTANT && p.ball == NLFEM_BALL_INFINITY)
        P.c = 3.0 / (4.0 * p.delta * p.delta * p.delta * p.delta);  // c_delta^inf (Sec. 3.3)
    else if (p.kernel == NLFEM_KERNEL_CONSTANT) P.c = 4.0 / (M_PI * p.delta * p.delta * p.delta * p.delta);
    else if (p.kernel == NLFEM_KERNEL_FRACTIONAL) P.c = (2.0 - 2.0 * p.s) / (M_PI * std::pow(p.delta, 2.0 - 2.0 * p.s));
    else if (p.kernel == NLFEM_KERNEL_TABULATED) P.c = 1.0;
    else P.c = 3.0 / (p.delta * p.delta * p.delta);
    if (p.kernel == NLFEM_KERNEL_TABULATED) {
        P.ntab = p.table_size;
        P.tinv = (double)(p.table_size - 1) / p.delta;
    }
    fill_rule(P.ro, p.quad_outer);
    fill_rule(P.ri, p.quad_inner);
    fill_gauss(P.dr, p.duffy_gauss);
    {
        // xi factor of the singular rule's integrand: Jacobian x D D^T x gamma's homogeneity
        // (gamma(xi z) = xi^alpha gamma(z), alpha = -2 - 2s, 0 for the constant kernel)
        const double alpha = p.kernel == NLFEM_KERNEL_FRACTIONAL ? -2.0 - 2.0 * p.s : 0.0;
        for (int c = 0; c < 3; ++c) P.dr.sxi[c] = 0.0;
        for (int i = 0; i < P.dr.n; ++i) {
            const double x = P.dr.x[i], w = P.dr.w[i];
            P.dr.sxi[0] += w * std::pow(x, 3.0 + alpha) * (1.0 - x) * (1.0 - x);  // identical
            P.dr.sxi[1] += w * std::pow(x, 4.0 + alpha) * (1.0 - x);              // common edge
            P.dr.sxi[2] += w * std::pow(x, 5.0 + alpha);                          // common vertex
        }
    }
    // Tab. 1: club for 0 < s < 1, diamond for -1 < s <= 0 (peridynamics: s = -1/2), heart for s <= -1
    if (p.close_rule == NLFEM_CLOSE_AUTO) {
        P.singular = p.kernel == NLFEM_KERNEL_FRACTIONAL;
        P.nozerodiv = p.kernel == NLFEM_KERNEL_PERIDYNAMIC;
    } else {
        P.singular = p.close_rule == NLFEM_CLOSE_DUFFY;
        P.nozerodiv = p.close_rule == NLFEM_CLOSE_NOZERODIV;
    }
    NLFEM_CHECK(!(P.singular && ndof == 2), NLFEM_ERR_UNSUPPORTED,
                "the singular rule is implemented for scalar kernels only");
    NLFEM_CHECK(!(P.singular && p.kernel == NLFEM_KERNEL_TABULATED), NLFEM_ERR_UNSUPPORTED,
                "the singular rule needs a homogeneous kernel; tabulated kernels take the standard rule");
    return P;
}

}  // namespace nlfem

using namespace nlfem;

struct nlfem_mesh_s {
    Mesh m;
};
struct nlfem_system_s {
    System s;
};
struct nlfem_batch_s {
    std::vector<std::unique_ptr<nlfem_system_s>> sys;
    std::vector<DBuf<double>> f;  // the load data, kept on the device
    std::vector<const double*> fptr;
    BatchExec exec;
    cudaStream_t cap = nullptr;   // capture stream (the legacy stream cannot be captured)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec_graph = nullptr;
    ~nlfem_batch_s() {
        if (exec_graph) cudaGraphExecDestroy(exec_graph);
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
    }
};

#define NLFEM_API_BEGIN try {
#define NLFEM_API_END                                   \
    }                                                   \
    catch (const ::nlfem::Error& e) {                   \
        set_error(e.msg);                               \
        return e.code;                                  \
    }                                                   \
    catch (const std::bad_alloc&) {                     \
        set_error("host allocation failed");            \
        return NLFEM_ERR_OOM;                           \
    }                                                   \
    catch (...) {                                       \
        set_error("unexpected exception");              \
        return NLFEM_ERR_CUDA;                          \
    }

extern "C" {

const char* nlfem_last_error(void) { return g_err.c_str(); }

const char* nlfem_version(void) { return "nlfem-gb300 0.1 (sm_103a)"; }

void nlfem_params_default(nlfem_params* p, int kernel) {
    if (!p) return;
    p->kernel = kernel;
    p->delta = 0.1;
    p->s = 0.5;
    p->kconst = NAN;
    p->ball = NLFEM_BALL_NOCAPS;
    p->quad_outer = 7;
    p->quad_inner = 7;
    p->duffy_gauss = 5;
    p->close_rule = NLFEM_CLOSE_AUTO;
    p->precision = NLFEM_PREC_FP64;
    p->mem_budget_bytes = 0;
    p->n_materials = 0;
    p->material_scale = nullptr;
    p->singular_precision = NLFEM_SINGULAR_FP64;
    p->geometry_precision = NLFEM_GEOMETRY_FP32;
    p->table_size = 0;
    p->kernel_table = nullptr;
}

// The library allocates its working buffers from the device's default memory pool
// (stream-ordered). Freed blocks are kept in the pool for the next assembly instead of
// being unmapped at every synchronisation (the pool's default); nlfem_trim_memory hands
// them back.
static void keep_pool_memory() {
    int dev = 0;
    NLFEM_CUDA_TRY(cudaGetDevice(&dev));
    static std::mutex mu;
    static std::vector<int> done;
    std::lock_guard<std::mutex> g(mu);
    if (std::find(done.begin(), done.end(), dev) != done.end()) return;
    cudaMemPool_t pool;
    NLFEM_CUDA_TRY(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t keep = UINT64_MAX;
    NLFEM_CUDA_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    done.push_back(dev);
}

int nlfem_trim_memory(void* stream) {
    NLFEM_API_BEGIN
    set_error("");
    int dev = 0;
    NLFEM_CUDA_TRY(cudaGetDevice(&dev));
    NLFEM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    cudaMemPool_t pool;
    NLFEM_CUDA_TRY(cudaDeviceGetDefaultMemPool(&pool, dev));
    NLFEM_CUDA_TRY(cudaMemPoolTrimTo(pool, 0));
    return NLFEM_OK;
    NLFEM_API_END
}

int nlfem_mesh_create(const double* verts, int64_t M, const int32_t* elems, int64_t K,
                      const int8_t* elem_label, int ndof_per_node, void* stream, nlfem_mesh_t* out) {
    NLFEM_API_BEGIN
    set_error("");
    NLFEM_CHECK(out != nullptr, NLFEM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    NLFEM_CHECK(verts && elems, NLFEM_ERR_INVALID_ARG, "verts and elems must not be NULL");
    NLFEM_CHECK(M >= 3 && K >= 1, NLFEM_ERR_INVALID_ARG, "need M >= 3 vertices and K >= 1 triangles");
    NLFEM_CHECK(M < (1ll << 31) && K < (1ll << 31) / 3, NLFEM_ERR_UNSUPPORTED, "mesh too large for 32-bit indices");
    NLFEM_CHECK(ndof_per_node == 1 || ndof_per_node == 2, NLFEM_ERR_INVALID_ARG, "ndof_per_node must be 1 or 2");
    cudaStream_t st = (cudaStream_t)stream;
    keep_pool_memory();
    nlfem_mesh_s* h = new nlfem_mesh_s();
    try {
        Mesh& m = h->m;
        m.M = M;
        m.K = K;
        m.ndof = ndof_per_node;
        upload(m.X, verts, (size_t)M, st);
        DBuf<int> T3;
        upload(T3, elems, (size_t)(3 * K), st);
        DBuf<int8_t> lab;
        if (elem_label) upload(lab, elem_label, (size_t)K, st);
        mesh_prepare(m, T3.p, elem_label ? lab.p : nullptr, st);
        NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
    } catch (...) {
        delete h;
        throw;
    }
    *out = h;
    return NLFEM_OK;
    NLFEM_API_END
}

int nlfem_mesh_create_dg(const double* verts, int64_t M, const int32_t* elems, int64_t K,
                         const int8_t* elem_label, int ndof_per_node, void* stream, nlfem_mesh_t* out) {
    NLFEM_API_BEGIN
    set_error("");
    NLFEM_CHECK(out != nullptr, NLFEM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    NLFEM_CHECK(verts && elems, NLFEM_ERR_INVALID_ARG, "verts and elems must not be NULL");
    NLFEM_CHECK(M >= 3 && K >= 1, NLFEM_ERR_INVALID_ARG, "need M >= 3 vertices and K >= 1 triangles");
    NLFEM_CHECK(M < (1ll << 31) && K < (1ll << 31) / 3, NLFEM_ERR_UNSUPPORTED, "mesh too large for 32-bit indices");
    NLFEM_CHECK(ndof_per_node == 1 || ndof_per_node == 2, NLFEM_ERR_INVALID_ARG, "ndof_per_node must be 1 or 2");
    cudaStream_t st = (cudaStream_t)stream;
    keep_pool_memory();
    nlfem_mesh_s* h = new nlfem_mesh_s();
    try {
        Mesh& m = h->m;
        m.K = K;
        m.ndof = ndof_per_node;
        DBuf<double2> X;
        upload(X, verts, (size_t)M, st);
        DBuf<int> T3;
        upload(T3, elems, (size_t)(3 * K), st);
        DBuf<int8_t> lab;
        if (elem_label) upload(lab, elem_label, (size_t)K, st);
        mesh_make_dg(m, X.p, M, T3.p, elem_label ? lab.p : nullptr, st);
    } catch (...) {
        delete h;
        throw;
    }
    *out = h;
    return NLFEM_OK;
    NLFEM_API_END
}

void nlfem_mesh_destroy(nlfem_mesh_t mesh) {
    if (!mesh) return;
    mesh->m.cache.reset();
    delete mesh;
}

int64_t nlfem_mesh_device_bytes(nlfem_mesh_t mesh) { return mesh ? mesh->m.device_bytes() : 0; }

int nlfem_mesh_set_materials(nlfem_mesh_t mesh, const int8_t* material, void* stream) {
    NLFEM_API_BEGIN
    set_error("");
    NLFEM_CHECK(mesh != nullptr, NLFEM_ERR_INVALID_ARG, "NULL mesh");
    Mesh& m = mesh->m;
    cudaStream_t st = (cudaStream_t)stream;
    if (!material) {
        m.mat.release();
        m.mat_max = -1;
        return NLFEM_OK;
    }
    std::vector<int8_t> h((size_t)m.K);
    NLFEM_CUDA_TRY(cudaMemcpyAsync(h.data(), material, (size_t)m.K,
                                   is_device_ptr(material) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, st));
    NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
    int mx = -1;
    for (int8_t v : h) {
        NLFEM_CHECK(v >= 0 && v < 16, NLFEM_ERR_INVALID_ARG, "material labels must be in 0..15");
        mx = v > mx ? v : mx;
    }
    upload(m.mat, h.data(), (size_t)m.K, st);
    NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
    m.mat_max = mx;
    return NLFEM_OK;
    NLFEM_API_END
}

int nlfem_mesh_pairs(nlfem_mesh_t mesh, const int32_t** k, const int32_t** l, int64_t* npairs) {
    NLFEM_API_BEGIN
    NLFEM_CHECK(mesh && k && l && npairs, NLFEM_ERR_INVALID_ARG, "NULL argument");
    NLFEM_CHECK(mesh->m.cache != nullptr, NLFEM_ERR_INVALID_ARG, "no pair list yet: call nlfem_assemble first");
    *k = mesh->m.cache->pk.p;
    *l = mesh->m.cache->pl.p;
    *npairs = mesh->m.cache->npairs;
    return NLFEM_OK;
    NLFEM_API_END
}

// The pair list, pattern and accumulation index of (mesh, delta, ball, outer rule, close
// rule), built unless the mesh handle holds them already.
static std::shared_ptr<PairCache> ensure_cache(Mesh& m, const Params& P, cudaStream_t st, cudaEvent_t* ev,
                                               double& t_pairs, double& t_pattern, bool& cached) {
    std::shared_ptr<PairCache> pc = m.cache;
    cached = pc && pc->delta == P.delta && pc->ball == P.ball && pc->nqo == P.ro.n && pc->ndof == P.ndof &&
             pc->close_mode == close_mode(P);
    t_pairs = t_pattern = 0;
    if (cached) return pc;
    m.cache.reset();
    pc = std::make_shared<PairCache>();
    pc->delta = P.delta;
    pc->ball = P.ball;
    pc->nqo = P.ro.n;
    pc->ndof = P.ndof;
    pc->close_mode = close_mode(P);
    NLFEM_CUDA_TRY(cudaEventRecord(ev[0], st));
    build_pairs(m, P, *pc, st);
    order_cut_pairs(m, *pc, P, st);
    NLFEM_CUDA_TRY(cudaEventRecord(ev[1], st));
    build_pattern(m, *pc, st);
    build_bulk_index(m, *pc, st);
    NLFEM_CUDA_TRY(cudaEventRecord(ev[2], st));
    NLFEM_CUDA_TRY(cudaEventSynchronize(ev[2]));
    t_pairs = elapsed_ms(ev[0], ev[1]);
    t_pattern = elapsed_ms(ev[1], ev[2]);
    pc->t_pairs_ms = t_pairs;
    pc->t_pattern_ms = t_pattern;
    m.cache = pc;
    return pc;
}

// The tables of a user kernel and of a label-dependent kernel go to the device with the
// system; the system's parameters point at them (and at the mesh's material labels).
static void attach_tables(System& S, const nlfem_params& p, const Mesh& m, cudaStream_t st);

// The user kernel's table goes to the device into bufs; P points at it.
static void attach_table(Params& P, const nlfem_params& p, DBuf<double>& t64, DBuf<float>& t32, cudaStream_t st) {
    if (p.kernel != NLFEM_KERNEL_TABULATED) return;
    std::vector<float> f(p.table_size);
    for (int i = 0; i < p.table_size; ++i) f[i] = (float)p.kernel_table[i];
    upload(t64, p.kernel_table, (size_t)p.table_size, st);
    upload(t32, f.data(), (size_t)p.table_size, st);
    NLFEM_CUDA_TRY(cudaStreamSynchronize(st));  // f is a host temporary
    P.tab64 = t64.p;
    P.tab32 = t32.p;
}

static void attach_tables(System& S, const nlfem_params& p, const Mesh& m, cudaStream_t st) {
    // Tab. 1: discontinuous ansatz functions for s <= 1/2 only (the factored form of
    // eq. case-one-factoredOut is not admissible on intersecting pairs for s > 1/2)
    NLFEM_CHECK(!(m.dg && S.prm.singular && p.kernel == NLFEM_KERNEL_FRACTIONAL && p.s > 0.5),
                NLFEM_ERR_UNSUPPORTED,
                "a discontinuous ansatz takes singular kernels with s <= 1/2 only (Sec. 2.3.2, Tab. 1)");
    attach_table(S.prm, p, S.tab64, S.tab32, st);
    if (p.n_materials <= 0) return;
    NLFEM_CHECK(m.mat.p && m.mat_max >= 0, NLFEM_ERR_INVALID_ARG,
                "n_materials > 0 needs material labels (nlfem_mesh_set_materials)");
    NLFEM_CHECK(m.mat_max < p.n_materials, NLFEM_ERR_INVALID_ARG,
                "a material label is >= n_materials");
    const int n2 = p.n_materials * p.n_materials;
    std::vector<float> t32(n2);
    for (int i = 0; i < n2; ++i) t32[i] = (float)p.material_scale[i];
    upload(S.msc64, p.material_scale, (size_t)n2, st);
    upload(S.msc32, t32.data(), (size_t)n2, st);
    NLFEM_CUDA_TRY(cudaStreamSynchronize(st));  // t32 is a host temporary
    S.prm.nmat = p.n_materials;
    S.prm.mat = m.mat.p;
    S.prm.msc64 = S.msc64.p;
    S.prm.msc32 = S.msc32.p;
}

// device bytes an assembly of (m, pc, P) needs beyond what the mesh handle holds
static int64_t assembly_bytes(const Mesh& m, const PairCache& pc, const Params& P) {
    const int64_t NE = contrib_entries(P.ndof);
    const int64_t nc = P.ndof == 1 ? 1 : 3;
    const int64_t work = P.precision == NLFEM_PREC_FP32_BULK
                             ? pc.n_upper * nc * 8 + pc.nduffy * NE * 8 + pc.npairs * 6 * nc * 4
                             : pc.npairs * NE * 8;
    return work + pc.nnz * 8 + pc.N * 8;
}

static void fill_info(System& S, Mesh& m, const PairCache& pc, double t_pairs, double t_pattern, bool cached) {
    nlfem_assembly_info& I = S.info;
    std::memset(&I, 0, sizeof I);
    I.npairs = pc.npairs;
    I.pairs_separated = pc.counts[0];
    I.pairs_vertex = pc.counts[1];
    I.pairs_edge = pc.counts[2];
    I.pairs_identical = pc.counts[3];
    I.nnz = pc.nnz;
    I.device_bytes = m.device_bytes() + (int64_t)(S.val.bytes() + S.F.bytes());
    I.ms_pairs = t_pairs;
    I.ms_pattern = t_pattern;
    I.pairs_whole = pc.nwhole;
    I.n_upper = pc.n_upper;
    I.n_contrib = pc.ncontrib;
    I.cached = cached ? 1 : 0;
}

int nlfem_assemble(nlfem_mesh_t mesh, const nlfem_params* params, const double* f_nodal, void* stream,
                   nlfem_system_t* out) {
    NLFEM_API_BEGIN
    set_error("");
    NLFEM_CHECK(mesh && params && out, NLFEM_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    Mesh& m = mesh->m;
    cudaStream_t st = (cudaStream_t)stream;
    Params P = make_params(*params, m.ndof);
    cudaEvent_t ev[12];  // [0..5] phases, [6..11] the quadrature kernels
    for (int i = 0; i < 12; ++i) NLFEM_CUDA_TRY(cudaEventCreate(&ev[i]));
    struct EvGuard {
        cudaEvent_t* e;
        ~EvGuard() {
            for (int i = 0; i < 12; ++i) cudaEventDestroy(e[i]);
        }
    } guard{ev};
    double t_pairs = 0, t_pattern = 0;
    bool cached = false;
    std::shared_ptr<PairCache> pc = ensure_cache(m, P, st, ev, t_pairs, t_pattern, cached);
    const int64_t NE = contrib_entries(P.ndof);
    const int64_t need = assembly_bytes(m, *pc, P) + m.device_bytes();
    if (params->mem_budget_bytes > 0 && need > params->mem_budget_bytes)
        throw Error{NLFEM_ERR_BUDGET, "assembly needs " + std::to_string(need) + " device bytes, budget is " +
                                          std::to_string(params->mem_budget_bytes)};
    nlfem_system_s* h = new nlfem_system_s();
    try {
        System& S = h->s;
        S.mesh = &m;
        S.pc = pc;
        S.prm = P;
        attach_tables(S, *params, m, st);
        P = S.prm;
        S.N = pc->N;
        S.nnz = pc->nnz;
        S.val.alloc(pc->nnz, st);
        S.F.alloc(pc->N, st);
        if (P.precision != NLFEM_PREC_FP32_BULK) S.contrib64.alloc(pc->npairs * NE, st);
        DBuf<double> fdev;
        const double* fptr = nullptr;
        if (f_nodal) {
            if (is_device_ptr(f_nodal)) fptr = f_nodal;
            else {
                upload(fdev, f_nodal, (size_t)(m.M * P.ndof), st);
                fptr = fdev.p;
            }
        }
        NLFEM_CUDA_TRY(cudaEventRecord(ev[3], st));
        run_quadrature(m, *pc, P, S, st, ev + 6);
        NLFEM_CUDA_TRY(cudaEventRecord(ev[4], st));
        run_reduction(m, *pc, P, S, st);
        NLFEM_CUDA_TRY(cudaEventRecord(ev[5], st));
        run_load(m, P, fptr, S, st);
        int redo = 0;
        if (P.precision == NLFEM_PREC_FP32_BULK)
            NLFEM_CUDA_TRY(cudaMemcpyAsync(&redo, &S.fix.p->redo, sizeof redo, cudaMemcpyDeviceToHost, st));
        NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
        if (redo) {
            // the pilot's estimate of the largest value was off by more than the headroom:
            // the accumulation runs again with the scale of the exact value (rare)
            NLFEM_CUDA_TRY(cudaEventRecord(ev[3], st));
            bulk_redo(m, *pc, P, S, st, ev + 6);
            NLFEM_CUDA_TRY(cudaEventRecord(ev[4], st));
            run_reduction(m, *pc, P, S, st);
            NLFEM_CUDA_TRY(cudaEventRecord(ev[5], st));
            NLFEM_CUDA_TRY(cudaMemcpyAsync(&redo, &S.fix.p->redo, sizeof redo, cudaMemcpyDeviceToHost, st));
            NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
            NLFEM_CHECK(!redo, NLFEM_ERR_CUDA, "internal error: fixed-point scale did not settle");
        }
        // contributions are no longer needed once reduced
        S.contrib32.release();
        S.contrib64.release();
        S.acc.release();
        S.llrec.release();
        fill_info(S, m, *pc, t_pairs, t_pattern, cached);
        nlfem_assembly_info& I = S.info;
        I.ms_quadrature = elapsed_ms(ev[3], ev[4]);
        I.ms_close = elapsed_ms(ev[6], ev[7]);
        I.ms_whole = elapsed_ms(ev[8], ev[9]);
        I.ms_cut = elapsed_ms(ev[9], ev[10]);
        I.ms_sums = elapsed_ms(ev[10], ev[11]);
        I.ms_reduce = elapsed_ms(ev[4], ev[5]);
    } catch (...) {
        delete h;
        throw;
    }
    *out = h;
    return NLFEM_OK;
    NLFEM_API_END
}

int nlfem_batch_assemble(const nlfem_mesh_t* meshes, const nlfem_params* params, const double* const* f_nodal,
                         int n, void* stream, nlfem_system_t* out) {
    NLFEM_API_BEGIN
    set_error("");
    NLFEM_CHECK(meshes && params && out && n >= 0, NLFEM_ERR_INVALID_ARG, "NULL argument or n < 0");
    for (int i = 0; i < n; ++i) {
        out[i] = nullptr;
        NLFEM_CHECK(meshes[i] != nullptr, NLFEM_ERR_INVALID_ARG, "NULL mesh handle");
        for (int j = 0; j < i; ++j)
            NLFEM_CHECK(meshes[j] != meshes[i], NLFEM_ERR_INVALID_ARG,
                        "a mesh handle appears twice in one batch (its pair list belongs to one parameter set)");
    }
    if (n == 0) return NLFEM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t ev[12];
    for (int i = 0; i < 12; ++i) NLFEM_CUDA_TRY(cudaEventCreate(&ev[i]));
    struct EvGuard {
        cudaEvent_t* e;
        ~EvGuard() {
            for (int i = 0; i < 12; ++i) cudaEventDestroy(e[i]);
        }
    } guard{ev};
    std::vector<std::unique_ptr<nlfem_system_s>> hs(n);
    std::vector<Params> P(n);
    std::vector<std::shared_ptr<PairCache>> pcs(n);
    std::vector<double> tp(n), tq(n);
    std::vector<char> cached(n);
    std::vector<DBuf<double>> fdev(n);
    std::vector<const double*> fptr(n, nullptr);
    for (int i = 0; i < n; ++i) {
        Mesh& m = meshes[i]->m;
        P[i] = make_params(params[i], m.ndof);
        bool c = false;
        pcs[i] = ensure_cache(m, P[i], st, ev, tp[i], tq[i], c);
        cached[i] = c;
        const int64_t need = assembly_bytes(m, *pcs[i], P[i]) + m.device_bytes();
        if (params[i].mem_budget_bytes > 0 && need > params[i].mem_budget_bytes)
            throw Error{NLFEM_ERR_BUDGET, "batch item " + std::to_string(i) + " needs " + std::to_string(need) +
                                              " device bytes, budget is " + std::to_string(params[i].mem_budget_bytes)};
        hs[i].reset(new nlfem_system_s());
        System& S = hs[i]->s;
        S.mesh = &m;
        S.pc = pcs[i];
        S.prm = P[i];
        attach_tables(S, params[i], m, st);
        P[i] = S.prm;
        S.N = pcs[i]->N;
        S.nnz = pcs[i]->nnz;
        S.val.alloc(pcs[i]->nnz, st);
        S.F.alloc(pcs[i]->N, st);
        if (f_nodal && f_nodal[i]) {
            if (is_device_ptr(f_nodal[i])) fptr[i] = f_nodal[i];
            else {
                upload(fdev[i], f_nodal[i], (size_t)(m.M * P[i].ndof), st);
                fptr[i] = fdev[i].p;
            }
        }
    }
    // FP64 systems one by one; FP32-bulk systems with fused launches
    std::vector<BatchSys> bulk;
    NLFEM_CUDA_TRY(cudaEventRecord(ev[3], st));
    for (int i = 0; i < n; ++i) {
        Mesh& m = meshes[i]->m;
        System& S = hs[i]->s;
        if (P[i].precision == NLFEM_PREC_FP32_BULK) {
            bulk.push_back(BatchSys{&m, pcs[i].get(), P[i], &S});
            continue;
        }
        S.contrib64.alloc(pcs[i]->npairs * contrib_entries(P[i].ndof), st);
        run_quadrature(m, *pcs[i], P[i], S, st, ev + 6);
        run_reduction(m, *pcs[i], P[i], S, st);
        run_load(m, P[i], fptr[i], S, st);
        S.contrib64.release();
    }
    if (!bulk.empty()) run_bulk_batch(bulk, st, ev + 6);
    NLFEM_CUDA_TRY(cudaEventRecord(ev[4], st));
    std::vector<int> redo(n, 0);
    for (int i = 0; i < n; ++i) {
        if (P[i].precision != NLFEM_PREC_FP32_BULK) continue;
        Mesh& m = meshes[i]->m;
        System& S = hs[i]->s;
        run_reduction(m, *pcs[i], P[i], S, st);
        run_load(m, P[i], fptr[i], S, st);
        NLFEM_CUDA_TRY(cudaMemcpyAsync(&redo[i], &S.fix.p->redo, sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    NLFEM_CUDA_TRY(cudaEventRecord(ev[5], st));
    NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
    const double ms_q = elapsed_ms(ev[3], ev[4]), ms_r = elapsed_ms(ev[4], ev[5]);
    const bool any_bulk = !bulk.empty();
    for (int i = 0; i < n; ++i) {
        Mesh& m = meshes[i]->m;
        System& S = hs[i]->s;
        if (redo[i]) {
            bulk_redo(m, *pcs[i], P[i], S, st, ev + 6);
            run_reduction(m, *pcs[i], P[i], S, st);
            int again = 0;
            NLFEM_CUDA_TRY(cudaMemcpyAsync(&again, &S.fix.p->redo, sizeof again, cudaMemcpyDeviceToHost, st));
            NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
            NLFEM_CHECK(!again, NLFEM_ERR_CUDA, "internal error: fixed-point scale did not settle");
        }
        S.contrib32.release();
        S.acc.release();
        S.llrec.release();
        fill_info(S, m, *pcs[i], tp[i], tq[i], cached[i] != 0);
        // times of the whole batch: the fused launches serve every system
        S.info.ms_quadrature = ms_q;
        S.info.ms_reduce = ms_r;
        if (any_bulk) {
            S.info.ms_close = elapsed_ms(ev[6], ev[7]);
            S.info.ms_whole = elapsed_ms(ev[8], ev[9]);
            S.info.ms_cut = elapsed_ms(ev[9], ev[10]);
            S.info.ms_sums = elapsed_ms(ev[10], ev[11]);
        }
    }
    for (int i = 0; i < n; ++i) out[i] = hs[i].release();
    return NLFEM_OK;
    NLFEM_API_END
}

// redo flags of the plan's systems after a run, and the redo of the flagged ones (rare)
static void batch_settle(nlfem_batch_s& b, cudaStream_t st, cudaEvent_t* ev) {
    const size_t n = b.exec.items.size();
    std::vector<int> redo(n, 0);
    for (size_t i = 0; i < n; ++i)
        NLFEM_CUDA_TRY(cudaMemcpyAsync(&redo[i], &b.exec.items[i].sys->fix.p->redo, sizeof(int),
                                       cudaMemcpyDeviceToHost, st));
    NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
    for (size_t i = 0; i < n; ++i) {
        if (!redo[i]) continue;
        BatchSys& it = b.exec.items[i];
        bulk_redo(*it.m, *it.pc, it.prm, *it.sys, st, ev);
        run_reduction(*it.m, *it.pc, it.prm, *it.sys, st);
        int again = 0;
        NLFEM_CUDA_TRY(cudaMemcpyAsync(&again, &it.sys->fix.p->redo, sizeof again, cudaMemcpyDeviceToHost, st));
        NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
        NLFEM_CHECK(!again, NLFEM_ERR_CUDA, "internal error: fixed-point scale did not settle");
    }
}

int nlfem_batch_create(const nlfem_mesh_t* meshes, const nlfem_params* params, const double* const* f_nodal,
                       int n, void* stream, nlfem_batch_t* out) {
    NLFEM_API_BEGIN
    set_error("");
    NLFEM_CHECK(meshes && params && out && n >= 1, NLFEM_ERR_INVALID_ARG, "NULL argument or n < 1");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        NLFEM_CHECK(meshes[i] != nullptr, NLFEM_ERR_INVALID_ARG, "NULL mesh handle");
        NLFEM_CHECK(params[i].precision == NLFEM_PREC_FP32_BULK, NLFEM_ERR_UNSUPPORTED,
                    "a batch plan holds FP32-bulk assemblies only");
        for (int j = 0; j < i; ++j)
            NLFEM_CHECK(meshes[j] != meshes[i], NLFEM_ERR_INVALID_ARG, "a mesh handle appears twice in one batch");
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t ev[12];
    for (int i = 0; i < 12; ++i) NLFEM_CUDA_TRY(cudaEventCreate(&ev[i]));
    struct EvGuard {
        cudaEvent_t* e;
        ~EvGuard() {
            for (int i = 0; i < 12; ++i) cudaEventDestroy(e[i]);
        }
    } guard{ev};
    std::unique_ptr<nlfem_batch_s> b(new nlfem_batch_s());
    b->sys.resize(n);
    b->f.resize(n);
    b->fptr.assign(n, nullptr);
    std::vector<double> tp(n), tq(n);
    std::vector<char> cached(n);
    for (int i = 0; i < n; ++i) {
        Mesh& m = meshes[i]->m;
        Params P = make_params(params[i], m.ndof);
        bool c = false;
        std::shared_ptr<PairCache> pc = ensure_cache(m, P, st, ev, tp[i], tq[i], c);
        cached[i] = c;
        const int64_t need = assembly_bytes(m, *pc, P) + m.device_bytes();
        if (params[i].mem_budget_bytes > 0 && need > params[i].mem_budget_bytes)
            throw Error{NLFEM_ERR_BUDGET, "batch item " + std::to_string(i) + " needs " + std::to_string(need) +
                                              " device bytes, budget is " + std::to_string(params[i].mem_budget_bytes)};
        b->sys[i].reset(new nlfem_system_s());
        System& S = b->sys[i]->s;
        S.mesh = &m;
        S.pc = pc;
        S.prm = P;
        attach_tables(S, params[i], m, st);
        P = S.prm;
        S.N = pc->N;
        S.nnz = pc->nnz;
        S.val.alloc(pc->nnz, st);
        S.F.alloc(pc->N, st);
        if (f_nodal && f_nodal[i]) {
            upload(b->f[i], f_nodal[i], (size_t)(m.M * P.ndof), st);  // copied: the plan owns its load data
            b->fptr[i] = b->f[i].p;
        }
        b->exec.items.push_back(BatchSys{&m, pc.get(), P, &S});
    }
    b->exec.prepare(st);
    b->exec.record(st, nullptr, true, b->fptr);
    batch_settle(*b, st, ev + 6);
    // capture the value assembly once; runs replay it
    NLFEM_CUDA_TRY(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    NLFEM_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    try {
        b->exec.record(b->cap, nullptr, true, b->fptr);
    } catch (...) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(b->cap, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    NLFEM_CUDA_TRY(cudaStreamEndCapture(b->cap, &b->graph));
    NLFEM_CUDA_TRY(cudaGraphInstantiate(&b->exec_graph, b->graph, 0));
    for (int i = 0; i < n; ++i) {
        System& S = b->sys[i]->s;
        fill_info(S, meshes[i]->m, *S.pc, tp[i], tq[i], cached[i] != 0);
    }
    *out = b.release();
    return NLFEM_OK;
    NLFEM_API_END
}

int nlfem_batch_run(nlfem_batch_t b, void* stream, double* ms) {
    NLFEM_API_BEGIN
    set_error("");
    NLFEM_CHECK(b != nullptr, NLFEM_ERR_INVALID_ARG, "NULL batch");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t ev[8];
    for (int i = 0; i < 8; ++i) NLFEM_CUDA_TRY(cudaEventCreate(&ev[i]));
    struct EvGuard {
        cudaEvent_t* e;
        ~EvGuard() {
            for (int i = 0; i < 8; ++i) cudaEventDestroy(e[i]);
        }
    } guard{ev};
    NLFEM_CUDA_TRY(cudaEventRecord(ev[6], st));
    NLFEM_CUDA_TRY(cudaGraphLaunch(b->exec_graph, st));
    NLFEM_CUDA_TRY(cudaEventRecord(ev[7], st));
    batch_settle(*b, st, ev);
    if (ms) *ms = elapsed_ms(ev[6], ev[7]);
    return NLFEM_OK;
    NLFEM_API_END
}

int nlfem_batch_system(nlfem_batch_t b, int i, nlfem_system_t* out) {
    NLFEM_API_BEGIN
    set_error("");
    NLFEM_CHECK(b && out && i >= 0 && i < (int)b->sys.size(), NLFEM_ERR_INVALID_ARG, "bad batch or index");
    *out = b->sys[i].get();
    return NLFEM_OK;
    NLFEM_API_END
}

void nlfem_batch_destroy(nlfem_batch_t b) { delete b; }

int nlfem_autotune(nlfem_mesh_t mesh, const nlfem_params* params, void* stream, int32_t best[2]) {
    NLFEM_API_BEGIN
    set_error("");
    NLFEM_CHECK(mesh && params && best, NLFEM_ERR_INVALID_ARG, "NULL argument");
    NLFEM_CHECK(params->precision == NLFEM_PREC_FP32_BULK, NLFEM_ERR_UNSUPPORTED,
                "the autotuner sets the FP32-bulk launch shapes");
    Mesh& m = mesh->m;
    cudaStream_t st = (cudaStream_t)stream;
    Params P = make_params(*params, m.ndof);
    DBuf<double> t64;
    DBuf<float> t32;
    attach_table(P, *params, t64, t32, st);
    cudaEvent_t ev[12];
    for (int i = 0; i < 12; ++i) NLFEM_CUDA_TRY(cudaEventCreate(&ev[i]));
    struct EvGuard {
        cudaEvent_t* e;
        ~EvGuard() {
            for (int i = 0; i < 12; ++i) cudaEventDestroy(e[i]);
        }
    } guard{ev};
    double tp = 0, tq = 0;
    bool cached = false;
    std::shared_ptr<PairCache> pc = ensure_cache(m, P, st, ev, tp, tq, cached);
    // scratch accumulators: the values are discarded, the launches are the real ones
    const int NC = pc->ndof == 1 ? 1 : 3;
    DBuf<unsigned long long> acc;
    DBuf<float> llrec;
    DBuf<FixState> fix;
    acc.alloc(std::max<int64_t>(pc->n_upper * NC, 1), st);
    llrec.alloc(std::max<int64_t>(pc->npairs * 6 * NC, 1), st);
    fix.alloc(1, st);
    fix.zero(st);
    pick_scale(m, *pc, P, fix.p, st);  // the real scale, so that the atomics are the real ones too
    const int cand[] = {2, 4, 8, 16, 32, 64};
    const int maxc = fast_max_chunk(P);
    for (int list = 0; list < 2; ++list) {
        const int64_t key = fast_tune_key(P, list);
        double best_ms = 1e300;
        int best_c = fast_blocks_per_sm(key), best_k = fast_chunk(key);
        // the cut-pair kernel also tries smaller chunks of outer points (shorter drains, more of
        // them); the whole-pair kernel has no chunks
        const int chunks[3] = {maxc, (maxc + 1) / 2, 2};
        for (int ci = 0; ci < (list == 1 ? 3 : 1); ++ci) {
            for (int c : cand) {
                set_fast_shape(key, c, list == 1 ? chunks[ci] : 0);
                double t = 1e300;
                for (int rep = 0; rep < 2; ++rep) {
                    NLFEM_CUDA_TRY(cudaEventRecord(ev[0], st));
                    launch_trunc_fast(m, *pc, P, BulkAcc{acc.p, llrec.p, &fix.p->scale, &fix.p->max_exact, 1}, st,
                                      ev + 2);
                    NLFEM_CUDA_TRY(cudaEventRecord(ev[1], st));
                    NLFEM_CUDA_TRY(cudaEventSynchronize(ev[1]));
                    t = std::min(t, elapsed_ms(ev[2 + list], ev[3 + list]));
                }
                if (t < best_ms) {
                    best_ms = t;
                    best_c = c;
                    best_k = list == 1 ? chunks[ci] : 0;
                }
            }
        }
        set_fast_shape(key, best_c, best_k);
        best[list] = best_c;
        if (list == 1) best[2] = best_k;
    }
    return NLFEM_OK;
    NLFEM_API_END
}

int nlfem_tune_set(const nlfem_params* params, const int32_t shape[3]) {
    NLFEM_API_BEGIN
    set_error("");
    NLFEM_CHECK(params && shape, NLFEM_ERR_INVALID_ARG, "NULL argument");
    const int ndof = params->kernel == NLFEM_KERNEL_PERIDYNAMIC ? 2 : 1;
    Params P = make_params(*params, ndof);
    NLFEM_CHECK(P.precision == NLFEM_PREC_FP32_BULK, NLFEM_ERR_UNSUPPORTED, "launch shapes apply to FP32 bulk");
    for (int i = 0; i < 2; ++i)
        NLFEM_CHECK(shape[i] >= 1 && shape[i] <= 64, NLFEM_ERR_INVALID_ARG, "blocks per SM must be in 1..64");
    NLFEM_CHECK(shape[2] >= 0 && shape[2] <= fast_max_chunk(P), NLFEM_ERR_INVALID_ARG,
                "outer points per chunk must be in 0.." + std::to_string(fast_max_chunk(P)));
    set_fast_shape(fast_tune_key(P, 0), shape[0], 0);
    set_fast_shape(fast_tune_key(P, 1), shape[1], shape[2]);
    return NLFEM_OK;
    NLFEM_API_END
}

int nlfem_system_csr(nlfem_system_t sys, const int64_t** row_ptr, const int32_t** col, const double** val,
                     int64_t* nrows, int64_t* nnz) {
    NLFEM_API_BEGIN
    NLFEM_CHECK(sys != nullptr, NLFEM_ERR_INVALID_ARG, "NULL system");
    PairCache* pc = sys->s.pc.get();
    if (row_ptr) *row_ptr = pc->row_ptr.p;
    if (col) *col = pc->col.p;
    if (val) *val = sys->s.val.p;
    if (nrows) *nrows = sys->s.N;
    if (nnz) *nnz = sys->s.nnz;
    return NLFEM_OK;
    NLFEM_API_END
}

int nlfem_system_rhs(nlfem_system_t sys, const double** F) {
    NLFEM_API_BEGIN
    NLFEM_CHECK(sys && F, NLFEM_ERR_INVALID_ARG, "NULL argument");
    *F = sys->s.F.p;
    return NLFEM_OK;
    NLFEM_API_END
}

int nlfem_system_dirichlet(nlfem_system_t sys, const int8_t** flags) {
    NLFEM_API_BEGIN
    NLFEM_CHECK(sys && flags, NLFEM_ERR_INVALID_ARG, "NULL argument");
    *flags = sys->s.mesh->dir.p;
    return NLFEM_OK;
    NLFEM_API_END
}

int nlfem_system_info(nlfem_system_t sys, nlfem_assembly_info* info) {
    NLFEM_API_BEGIN
    NLFEM_CHECK(sys && info, NLFEM_ERR_INVALID_ARG, "NULL argument");
    *info = sys->s.info;
    return NLFEM_OK;
    NLFEM_API_END
}

int nlfem_solve(nlfem_system_t sys, const double* g_nodal, double tol_rel, int max_iter, double* u_out,
                nlfem_solve_info* info, void* stream) {
    NLFEM_API_BEGIN
    set_error("");
    NLFEM_CHECK(sys && u_out, NLFEM_ERR_INVALID_ARG, "NULL argument");
    NLFEM_CHECK(tol_rel > 0 && max_iter > 0, NLFEM_ERR_INVALID_ARG, "need tol_rel > 0 and max_iter > 0");
    NLFEM_CHECK(is_device_ptr(u_out), NLFEM_ERR_INVALID_ARG, "u_out must be device memory");
    cudaStream_t st = (cudaStream_t)stream;
    DBuf<double> gdev;
    const double* g = nullptr;
    if (g_nodal) {
        if (is_device_ptr(g_nodal)) g = g_nodal;
        else {
            upload(gdev, g_nodal, (size_t)sys->s.N, st);
            g = gdev.p;
        }
    }
    return solve_system(sys->s, g, tol_rel, max_iter, u_out, info, st);
    NLFEM_API_END
}

int nlfem_solve_neumann(nlfem_system_t sys, double tol_rel, int max_iter, double* u_out, nlfem_solve_info* info,
                        void* stream) {
    NLFEM_API_BEGIN
    set_error("");
    NLFEM_CHECK(sys && u_out, NLFEM_ERR_INVALID_ARG, "NULL argument");
    NLFEM_CHECK(tol_rel > 0 && max_iter > 0, NLFEM_ERR_INVALID_ARG, "need tol_rel > 0 and max_iter > 0");
    NLFEM_CHECK(is_device_ptr(u_out), NLFEM_ERR_INVALID_ARG, "u_out must be device memory");
    return solve_neumann(sys->s, tol_rel, max_iter, u_out, info, (cudaStream_t)stream);
    NLFEM_API_END
}

int nlfem_system_census(nlfem_system_t sys, int64_t counts[16], void* stream) {
    NLFEM_API_BEGIN
    NLFEM_CHECK(sys && counts, NLFEM_ERR_INVALID_ARG, "NULL argument");
    run_census(*sys->s.mesh, *sys->s.pc, sys->s.prm, counts, (cudaStream_t)stream);
    return NLFEM_OK;
    NLFEM_API_END
}

void nlfem_system_destroy(nlfem_system_t sys) { delete sys; }

}  // extern "C"
