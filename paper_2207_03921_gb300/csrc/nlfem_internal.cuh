// Internal declarations of the nlfem CUDA library (sm_103a).
// The public C ABI is include/nlfem.h; everything here is private to the .so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <vector>

#include "../../include/nlfem.h"

// ------------------------------------------------------------------------------------------
// errors
// ------------------------------------------------------------------------------------------
namespace nlfem {

void set_error(const std::string& msg);

struct Error {
    int code;
    std::string msg;
};

#define NLFEM_CUDA_TRY(expr)                                                                  \
    do {                                                                                      \
        cudaError_t e__ = (expr);                                                             \
        if (e__ != cudaSuccess)                                                               \
            throw ::nlfem::Error{NLFEM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e__)}; \
    } while (0)

#define NLFEM_CHECK(cond, code, msg)                                                           \
    do {                                                                                      \
        if (!(cond)) throw ::nlfem::Error{(code), (msg)};                                     \
    } while (0)

#define NLFEM_LAUNCH_CHECK() NLFEM_CUDA_TRY(cudaGetLastError())

// stream-ordered device buffer
template <typename T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaStream_t s = 0;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept : p(o.p), n(o.n), s(o.s) {
        o.p = nullptr;
        o.n = 0;
    }
    DBuf& operator=(DBuf&& o) noexcept {
        if (this != &o) {
            release();
            p = o.p;
            n = o.n;
            s = o.s;
            o.p = nullptr;
            o.n = 0;
        }
        return *this;
    }
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        n = 0;
    }
    void alloc(size_t count, cudaStream_t st) {
        release();
        s = st;
        n = count;
        if (count == 0) return;
        cudaError_t e = cudaMallocAsync((void**)&p, count * sizeof(T), st);
        if (e != cudaSuccess) {
            p = nullptr;
            n = 0;
            (void)cudaGetLastError();
            throw Error{NLFEM_ERR_OOM, "device allocation of " + std::to_string(count * sizeof(T)) + " bytes failed"};
        }
    }
    void zero(cudaStream_t st) {
        if (n) NLFEM_CUDA_TRY(cudaMemsetAsync(p, 0, n * sizeof(T), st));
    }
    size_t bytes() const { return n * sizeof(T); }
    // keep the buffer if it already has count elements (no stream operation then)
    void ensure(size_t count, cudaStream_t st) {
        if (p && n == count) return;
        alloc(count, st);
    }
    void swap_with(DBuf& o) {
        std::swap(p, o.p);
        std::swap(n, o.n);
        std::swap(s, o.s);
    }
};

// ------------------------------------------------------------------------------------------
// mesh and system handles
// ------------------------------------------------------------------------------------------
struct PairCache;

// Everything the bulk quadrature reads of an element, in one 48-byte record (three 16-byte
// loads): vertex 0 in FP64, the FP32 edge vectors, the nodes and |det J| in FP32.
struct __align__(16) ElemRec {
    double2 v0;
    float4 E;        // (v1 - v0, v2 - v0)
    int n0, n1, n2;  // counter-clockwise
    float det;
};
static_assert(sizeof(ElemRec) == 48, "ElemRec is three 16-byte words");

struct Mesh {
    int64_t M = 0, K = 0;
    int ndof = 1;
    DBuf<double2> X;      // vertices [M]
    DBuf<int4> T;         // CCW triangles [K] (w unused)
    DBuf<double> det;     // |det J_k| = 2 |E_k| [K]
    DBuf<int8_t> lab;     // element label, 1 = Omega [K]
    DBuf<int8_t> dir;     // node is Dirichlet [M]
    DBuf<int> ne_ptr;     // node -> elements CSR [M + 1]
    DBuf<int> ne_idx;     // [3K], sorted per node
    double bbox[4] = {0, 0, 0, 0};  // xmin, ymin, xmax, ymax
    double rmax = 0;      // max element radius (centroid to vertex)
    DBuf<double2> cen;    // centroids [K]
    DBuf<float4> E32;     // FP32 edge vectors (v1 - v0, v2 - v0) [K], each rounded once from FP64
    DBuf<float> det32;    // |det J_k| in FP32 [K]
    DBuf<ElemRec> rec;    // packed element records [K]
    DBuf<double> rad;     // radii [K]
    DBuf<int8_t> mat;     // material labels of a label-dependent kernel [K] (empty: none)
    // discontinuous ansatz: every element has its own copies of its vertices (nodes 3k + a);
    // Tpos holds the original vertex ids, which classify the pairs (shared vertices as points)
    bool dg = false;
    DBuf<int4> Tpos;
    const int4* tpos() const { return Tpos.p ? Tpos.p : T.p; }
    int mat_max = -1;     // largest material label
    std::shared_ptr<PairCache> cache;  // pair list, pattern and slot index of the last (delta, ball, rule)
    int64_t device_bytes() const;
};

// rule table passed by value to the kernels
struct Rule {
    int n;
    double l[16][3];
    double w[16];
};

struct DuffyRule {
    int n;
    double x[32], w[32];
    double sum_w, sum_wx;  // sums of the 1D rule (exact 1 and 1/2 up to rounding)
    double sxi[3];         // xi sums of the singular rule: identical, edge, vertex (set with the kernel)
};

struct Params {
    int kernel, ball, close_rule, precision, ndof;
    double delta, delta2, s, c;
    Rule ro, ri;
    DuffyRule dr;
    bool singular;    // Tab. 1 club rule on intersecting pairs
    bool nozerodiv;   // Tab. 1 diamond rule on intersecting pairs
    // label-dependent kernel: factor msc[mat[k] * nmat + mat[l]] on pair (k, l); nmat = 0: none
    int nmat;
    const int8_t* mat;
    const double* msc64;
    const float* msc32;
    // user-defined radial kernel: g at r_i = i / tinv, i < ntab, on the device
    int ntab;
    double tinv;
    const double* tab64;
    const float* tab32;
    // FP32 bulk: the singular rule in FP32 (else FP64); every cut outer point cut in FP64
    int sing32;
    int geo64;
};

// g(r) of the tabulated kernel, r = sqrt(d2): linear between the table values, held beyond
template <typename R>
__device__ __forceinline__ R table_g(const R* __restrict__ tab, int n, R tinv, R d2) {
    const R t = sqrt(d2) * tinv;
    const int i = (int)t;
    if (i >= n - 1) return tab[n - 1];
    const R w = t - (R)i;
    return ((R)1 - w) * tab[i] + w * tab[i + 1];
}

// maximum of v over the warp, then one atomicMax per warp (every lane of the warp must call it)
__device__ __forceinline__ void warp_atomic_max(int* out, int v) {
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, v);
}
__device__ __forceinline__ void warp_atomic_max(unsigned long long* out, unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, v);
}

// kernel factor of the ordered pair (k, l) for label-dependent kernels
__device__ __forceinline__ double pair_factor64(const Params& P, int k, int l) {
    return P.nmat ? P.msc64[P.mat[k] * P.nmat + P.mat[l]] : 1.0;
}

struct FixState;

// Interaction graph, CSR pattern and reduction index of one (mesh, delta, ball, outer rule, ndof).
struct PairCache {
    double delta = -1;
    int ball = -1, nqo = -1, ndof = -1, close_mode = -1;  // close_mode: 0 standard, 1 singular, 2 diamond
    int64_t npairs = 0;
    DBuf<int64_t> pair_ptr;  // [K + 1]
    DBuf<int> pk, pl;        // [P], sorted by (k, l)
    DBuf<int8_t> pcls;       // shared vertex count [P]
    DBuf<int64_t> pT_ptr;    // [K + 1] pairs grouped by l
    DBuf<int> pT_id;         // [P] pair ids, sorted per l
    DBuf<int> duffy_ids;     // intersecting pairs under the singular or diamond rule, in pair order
    int64_t nduffy = 0;
    DBuf<int> whole_ids;     // pairs on the standard rule with E_l inside the ball of every point of E_k
    DBuf<int> cut_ids;       // the other pairs on the standard rule, ordered by fan-triangle count
    int64_t nwhole = 0, ncut = 0;
    int64_t counts[4] = {0, 0, 0, 0};  // separated, vertex, edge, identical
    // node-level pattern
    DBuf<int64_t> nrow_ptr;  // [M + 1]
    DBuf<int> ncol;          // [nnz_node]
    DBuf<int> ntpos;         // [nnz_node] rank of the row in the column's row (until the bulk index is built)
    int64_t nnz_node = 0;
    int max_row = 0;
    // dof-level CSR
    int64_t N = 0, nnz = 0;
    DBuf<int64_t> row_ptr;   // [N + 1]
    DBuf<int> col;           // [nnz]
    DBuf<int64_t> tpos;      // [nnz] position of the transposed entry
    DBuf<int64_t> seg_ptr;   // [nnz + 1] contribution segments per CSR slot (upper slots only)
    DBuf<uint64_t> idx;      // [ncontrib] packed ((pair - pbase[row]) << 6) | transposed << 5 | entry
    DBuf<int64_t> pbase;     // [M] first pair id a node row refers to
    int64_t ncontrib = 0;
    DBuf<int64_t> up_pos;    // node-level upper entries (i, j >= i): pattern position
    DBuf<int> up_row;        //   and row i (built with the slot index, for the ordered reduction)
    int64_t n_upper = 0;
    bool slots_built = false;
    // FP32 bulk: the fixed-point scale the pilot pass picked for the parameters with this key
    // (a function of the pattern and the parameters alone, so a later assembly reuses it)
    uint64_t scale_key = 0;
    bool scale_memo_valid = false;
    DBuf<FixState> scale_memo;
    // FP32-bulk accumulation index: upper entries numbered row by row in node order
    DBuf<int64_t> up_start;  // [M + 1] first upper entry of each node row
    DBuf<int> epos;          // [K * 8] upper entry of each node pair of an element (6 used)
    DBuf<uint16_t> klr_whole, klr_cut;  // [9][list length] rank of (k_a, l_b) in row min(k_a, l_b)
    DBuf<int2> kl_whole;                // [nwhole] the elements (k, l) of every whole-pair list entry
    int64_t acc_terms = 0;   // bound on the number of values added into one upper entry
    double t_pairs_ms = 0, t_pattern_ms = 0;
};

struct SolveState;

// Fixed-point scale of one FP32-bulk assembly, chosen on the device (no host round trip):
// a pilot pass records max_pilot, the scale 2^shift follows; the main pass records
// max_exact, and redo = 1 if shift could overflow a sum or wastes more than 2^16 of range.
struct FixState {
    unsigned int max_pilot;  // bits of a positive float
    unsigned int max_exact;
    int shift, shift_exact, redo, pad;
    float scale;             // 2^shift
    float pad2;
};

// S with terms * maxabs * 2^S <= 2^62 (headroom_bits more below that), from the exact binary
// exponent of maxabs * terms; the same function on the host and the device
__host__ __device__ inline int fix_shift(float maxabs, int64_t terms, int headroom_bits) {
    if (!(maxabs > 0.f)) return 0;
    const double x = (double)maxabs * (double)(terms > 0 ? terms : 1);  // exact: 24 + 40 bits < 53 + 11
    int e = 0;
    const double mant = frexp(x, &e);  // x = mant 2^e, mant in [0.5, 1)
    const int c = mant == 0.5 ? e - 1 : e;  // ceil(log2(x))
    const int S = 62 - c - headroom_bits;
    return S < -120 ? -120 : (S > 120 ? 120 : S);
}

struct System {
    Mesh* mesh = nullptr;
    std::shared_ptr<PairCache> pc;  // the pattern this system was assembled on
    Params prm;
    int64_t N = 0, nnz = 0;
    DBuf<double> val;        // [nnz]
    DBuf<double> F;          // [N]
    DBuf<float> contrib32;   // records [P * NE] (FP32 bulk: only the close-list pairs, in list order)
    DBuf<double> contrib64;  // records [P * NE] (FP64 plain)
    DBuf<unsigned long long> acc;  // FP32 bulk: fixed-point upper entries [n_upper * NC]
    DBuf<float> llrec;       // FP32 bulk: ll of every pair [P * 6 NC]
    DBuf<FixState> fix;      // FP32 bulk: the fixed-point scale
    DBuf<double> msc64;      // label-dependent kernel: the scale table on the device
    DBuf<float> msc32;
    DBuf<double> tab64;      // user-defined radial kernel: the table on the device
    DBuf<float> tab32;
    nlfem_assembly_info info;
    std::shared_ptr<SolveState> solver;
};

// ------------------------------------------------------------------------------------------
// host-side entry points of the translation units
// ------------------------------------------------------------------------------------------
void mesh_prepare(Mesh& m, const int* T3_dev, const int8_t* lab_dev, cudaStream_t st);
void mesh_make_dg(Mesh& m, const double2* X_dev, int64_t M_in, const int* T3_dev, const int8_t* lab_dev,
                  cudaStream_t st);
void build_pairs(Mesh& m, const Params& prm, PairCache& pc, cudaStream_t st);
void build_pattern(Mesh& m, PairCache& pc, cudaStream_t st);
// ev[0..5] are recorded on st: [0, 1] around the close-list kernel (singular or diamond
// rule), [2, 3] whole-pair kernel, [3, 4] cut-pair kernel (FP64: every pair), [4, 5] element
// sums and close-list adds
void run_quadrature(Mesh& m, PairCache& pc, const Params& prm, System& sys, cudaStream_t st, cudaEvent_t* ev);
void run_reduction(Mesh& m, PairCache& pc, const Params& prm, System& sys, cudaStream_t st);
void run_load(Mesh& m, const Params& prm, const double* f_nodal, System& sys, cudaStream_t st);
// per-pair contribution record: 21 scalar entries padded to 24, 84 peridynamic components
// padded to 88, so that in FP32 and FP64 a record covers whole 32-byte sectors
constexpr int NLFEM_REC1 = 24, NLFEM_REC2 = 88;
int64_t contrib_entries(int ndof);
void run_census(Mesh& m, PairCache& pc, const Params& prm, int64_t* out, cudaStream_t st);
// fixed-point accumulation of the FP32-bulk kernels; acc == nullptr: pilot pass that only
// records the largest |value| of every pstride-th pair
struct BulkAcc {
    unsigned long long* acc;
    float* llrec;           // [P][6 NC] per-pair ll records
    const float* scale_p;   // 2^S in device memory
    unsigned int* maxabs;
    int64_t pstride;
};
// FP32 bulk: after the quadrature, read FixState.redo (with the final synchronisation) and
// call bulk_redo if it is set
void bulk_redo(Mesh& m, PairCache& pc, const Params& prm, System& sys, cudaStream_t st, cudaEvent_t* ev);
// pilot pass and scale choice into f (f zeroed by the caller)
void pick_scale(Mesh& m, PairCache& pc, const Params& prm, FixState* f, cudaStream_t st);
void launch_trunc_fast(Mesh& m, PairCache& pc, const Params& prm, const BulkAcc& b, cudaStream_t st,
                       cudaEvent_t* ev);
// one request of a batched launch (all items of one call share the kernel class: kernel
// type, outer and inner rule, ball)
struct BulkItem {
    Mesh* m;
    PairCache* pc;
    Params prm;
    BulkAcc b;
};
// a fused launch over the items' pairs of one list (0 whole, 1 cut): the request table is
// uploaded by make_fused, run_fused only launches (capturable into a CUDA graph)
struct FusedLaunch;
std::shared_ptr<FusedLaunch> make_fused(const std::vector<BulkItem>& items, int list, int pilot, cudaStream_t st);
void run_fused(const FusedLaunch& f, cudaStream_t st);
void set_fast_attributes();  // shared-memory limits of the cut-pair kernels (once per device)
// grid size of the bulk launches: blocks per SM for (kernel class, list); set by the autotuner
int64_t fast_tune_key(const Params& prm, int list);
int fast_blocks_per_sm(int64_t key);
void set_fast_blocks_per_sm(int64_t key, int bps);
int fast_chunk(int64_t key);                       // 0 = the kernel's full chunk
void set_fast_shape(int64_t key, int bps, int chunk);
int fast_max_chunk(const Params& prm);             // outer points per chunk of the cut-pair kernel
// FP32-bulk assembly of several systems with fused bulk launches (quad.cu)
struct BatchSys {
    Mesh* m;
    PairCache* pc;
    Params prm;
    System* sys;
};
// The FP32-bulk value assembly of several systems: prepare() allocates the per-system
// working buffers and uploads the fused launches' request tables; record() enqueues every
// step (close lists, pilot, scale, fused bulk launches, ll sums, close-list adds, check, and with finish
// also the conversion to CSR and the load vector) with stream operations only, so that it can
// be captured into a CUDA graph and replayed.
struct BatchExec {
    std::vector<BatchSys> items;
    std::vector<std::shared_ptr<FusedLaunch>> pilot, whole, cut;
    void prepare(cudaStream_t st);
    void record(cudaStream_t st, cudaEvent_t* ev, bool finish, const std::vector<const double*>& f);
};
void run_bulk_batch(std::vector<BatchSys>& items, cudaStream_t st, cudaEvent_t* ev);
void build_bulk_index(Mesh& m, PairCache& pc, cudaStream_t st);
void build_slots(Mesh& m, PairCache& pc, cudaStream_t st);
void order_cut_pairs(Mesh& m, PairCache& pc, const Params& prm, cudaStream_t st);
inline int close_mode(const Params& P) { return P.singular ? 1 : (P.nozerodiv ? 2 : 0); }
int solve_system(System& S, const double* g, double tol, int max_iter, double* u_out, nlfem_solve_info* info,
                 cudaStream_t st);
int solve_neumann(System& S, double tol, int max_iter, double* u_out, nlfem_solve_info* info, cudaStream_t st);

// exclusive scan of int64 counts in place (n values -> n + 1 offsets in out)
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st);
// segmented sort of int keys (with an optional int payload) within [ptr[s], ptr[s + 1])
void segmented_sort_i32(int* keys, int* vals, const int64_t* ptr, int64_t nseg, int max_len,
                        cudaStream_t st);

double elapsed_ms(cudaEvent_t a, cudaEvent_t b);
// largest ptr[i + 1] - ptr[i] over i < n
int64_t max_segment_i64(const int64_t* ptr, int64_t n, cudaStream_t st);

}  // namespace nlfem

// rank of column hi among the columns >= lo of node row lo of the node-level pattern (the
// diagonal has rank 0); -1 if the column is missing
__device__ __forceinline__ int upper_rank(const int64_t* __restrict__ nptr, const int* __restrict__ ncol, int lo,
                                          int hi) {
    const int64_t b = nptr[lo], e = nptr[lo + 1];
    auto lower = [&](int v) {
        int64_t a = b, c = e;
        while (a < c) {
            const int64_t mid = (a + c) >> 1;
            if (ncol[mid] < v) a = mid + 1;
            else c = mid;
        }
        return a;
    };
    const int64_t ph = lower(hi), pd = lower(lo);
    if (ph >= e || ncol[ph] != hi || pd >= e || ncol[pd] != lo) return -1;
    return (int)(ph - pd);
}

// ------------------------------------------------------------------------------------------
// canonical FP64 geometry (shared by all kernels of this library)
//
// Every operation is an explicitly rounded IEEE operation (no FMA contraction), so
// the interaction decisions are the ones of the written-out arithmetic:
//   point on triangle:  x = (l0*v0 + l1*v1) + l2*v2
//   vertex in ball:     dx = vx - cx, dy = vy - cy, (dx*dx + dy*dy) <= delta*delta
//   edge crossings:     u = b - a, e = a - c, A = u.u, B = e.u, C = e.e - delta2,
//                       disc = B*B - A*C > 0, t = (-B -+ sqrt(disc)) / A in (0, 1);
//                       t < 1e-12 or t > 1 - 1e-12 means the circle passes through
//                       the edge's end vertex, which is emitted instead
//   cap centre:         q = Q - P, len = sqrt(q.q) > 1e-9 delta,
//                       m = (cx + delta*(qy/len), cy + delta*(-qx/len))
// (Sec. 2.2, Defs. 2.1 and 2.2, with the tie rules spelled out above).
// ------------------------------------------------------------------------------------------
#define NLFEM_TAU 1e-12
#define NLFEM_CAP_MIN 1e-9
#define NLFEM_MAXPOLY 16

struct CPt {
    double x, y;   // absolute coordinates
    double b1, b2; // barycentric coordinates w.r.t. the inner element (b0 = 1 - b1 - b2)
    int e;         // boundary edge index
    double t;      // parameter on that edge (0 for vertices)
    int vert;
};

__device__ __forceinline__ double2 nl_map(const double2 V[3], double l0, double l1, double l2) {
    double x = __dadd_rn(__dadd_rn(__dmul_rn(l0, V[0].x), __dmul_rn(l1, V[1].x)), __dmul_rn(l2, V[2].x));
    double y = __dadd_rn(__dadd_rn(__dmul_rn(l0, V[0].y), __dmul_rn(l1, V[1].y)), __dmul_rn(l2, V[2].y));
    return make_double2(x, y);
}

__device__ __forceinline__ double nl_d2(double2 v, double2 c) {
    double dx = __dsub_rn(v.x, c.x), dy = __dsub_rn(v.y, c.y);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

__device__ __forceinline__ bool nl_joined(const CPt& P, const CPt& Q) {
    if (Q.e == P.e && Q.t > P.t) return true;
    if (Q.vert && Q.e == (P.e + 1) % 3) return true;
    return false;
}

__device__ __forceinline__ void nl_push(CPt* raw, int& n, const CPt& c) {
    if (n > 0 && raw[n - 1].x == c.x && raw[n - 1].y == c.y) {
        if (raw[n - 1].vert && !c.vert) return;  // keep the vertex
        raw[n - 1] = c;                          // keep the later one
    } else if (n < NLFEM_MAXPOLY) {              // at most 6 points reach here (2 per edge)
        raw[n++] = c;
    }
}

// E_l = V cut by the ball approximation around c. Returns the number of polygon points
// written to out (with barycentric coordinates); full = all three vertices inside.
// With out == nullptr only the count is returned (interaction predicate).
__device__ __forceinline__ int nl_clip(const double2 V[3], double2 c, double delta, double delta2,
                                       bool caps, CPt* out, bool& full) {
    bool ins[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) ins[a] = nl_d2(V[a], c) <= delta2;
    if (ins[0] && ins[1] && ins[2]) {
        full = true;
        return 3;
    }
    full = false;
    CPt raw[NLFEM_MAXPOLY];
    int n = 0;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int eb = (e + 1) % 3;
        const double2 A_ = V[e], B_ = V[eb];
        const double bA1 = (e == 1) ? 1.0 : 0.0, bA2 = (e == 2) ? 1.0 : 0.0;
        const double bB1 = (eb == 1) ? 1.0 : 0.0, bB2 = (eb == 2) ? 1.0 : 0.0;
        if (ins[e]) nl_push(raw, n, CPt{A_.x, A_.y, bA1, bA2, e, 0.0, 1});
        double ux = __dsub_rn(B_.x, A_.x), uy = __dsub_rn(B_.y, A_.y);
        double ex = __dsub_rn(A_.x, c.x), ey = __dsub_rn(A_.y, c.y);
        double A = __dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy));
        double B = __dadd_rn(__dmul_rn(ex, ux), __dmul_rn(ey, uy));
        double C = __dsub_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), delta2);
        double disc = __dsub_rn(__dmul_rn(B, B), __dmul_rn(A, C));
        if (disc > 0.0) {
            double r = __dsqrt_rn(disc);
            double ts[2] = {__ddiv_rn(__dsub_rn(-B, r), A), __ddiv_rn(__dadd_rn(-B, r), A)};
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                double t = ts[j];
                if (!(t > 0.0 && t < 1.0)) continue;
                if (t < NLFEM_TAU) {
                    nl_push(raw, n, CPt{A_.x, A_.y, bA1, bA2, e, 0.0, 1});
                } else if (t > 1.0 - NLFEM_TAU) {
                    nl_push(raw, n, CPt{B_.x, B_.y, bB1, bB2, eb, 0.0, 1});
                } else {
                    double px = __dadd_rn(A_.x, __dmul_rn(t, ux));
                    double py = __dadd_rn(A_.y, __dmul_rn(t, uy));
                    // barycentric: (1 - t) at vertex e, t at vertex eb
                    double b1 = (e == 1 ? 1.0 - t : 0.0) + (eb == 1 ? t : 0.0);
                    double b2 = (e == 2 ? 1.0 - t : 0.0) + (eb == 2 ? t : 0.0);
                    nl_push(raw, n, CPt{px, py, b1, b2, e, t, 0});
                }
            }
        }
    }
    if (n >= 2 && raw[n - 1].x == raw[0].x && raw[n - 1].y == raw[0].y) {
        if (raw[n - 1].vert && !raw[0].vert) raw[0] = raw[n - 1];
        --n;
    }
    // inverse map of E_l for cap centres
    double ex1 = V[1].x - V[0].x, ey1 = V[1].y - V[0].y, ex2 = V[2].x - V[0].x, ey2 = V[2].y - V[0].y;
    double dj = ex1 * ey2 - ey1 * ex2;
    int m = 0;
    for (int i = 0; i < n && m < NLFEM_MAXPOLY; ++i) {
        if (out) out[m] = raw[i];
        ++m;
        if (caps && n >= 2 && m < NLFEM_MAXPOLY) {
            const CPt& P = raw[i];
            const CPt& Q = raw[(i + 1) % n];
            if (!nl_joined(P, Q)) {
                double qx = __dsub_rn(Q.x, P.x), qy = __dsub_rn(Q.y, P.y);
                double len = __dsqrt_rn(__dadd_rn(__dmul_rn(qx, qx), __dmul_rn(qy, qy)));
                if (len > NLFEM_CAP_MIN * delta) {
                    if (out) {
                        double mx = __dadd_rn(c.x, __dmul_rn(delta, __ddiv_rn(qy, len)));
                        double my = __dadd_rn(c.y, __dmul_rn(delta, __ddiv_rn(-qx, len)));
                        double px = mx - V[0].x, py = my - V[0].y;
                        double b1 = (px * ey2 - py * ex2) / dj;
                        double b2 = (ex1 * py - ey1 * px) / dj;
                        out[m] = CPt{mx, my, b1, b2, -1, 0.0, 0};
                    }
                    ++m;
                }
            }
        }
    }
    return m;
}

// ------------------------------------------------------------------------------------------
// Infinity norm ball (Sec. 2.2, Def. of the infinity norm ball): E_l cut exactly by the closed
// square |y - c|_inf <= delta. Canonical FP64 operation order, in coordinates relative to c:
//   p = (vx - cx, vy - cy) per vertex, each difference rounded once; full = every vertex has
//   |px| <= delta and |py| <= delta;
//   Sutherland-Hodgman passes by x <= delta, y <= delta, x >= -delta, y >= -delta (in this
//   order); half-plane (axis a, sign s): inside iff s * p[a] <= delta; a pass walks S -> E over
//   consecutive points from S = the last point, E = the first, and emits the crossing
//     t = (s delta - S[a]) / (E[a] - S[a]),  X[a] = s delta,  X[b] = S[b] + t (E[b] - S[b])
//   where S and E lie on different sides, then E if E is inside;
//   consecutive points that coincide exactly (also the last and the first) are merged;
//   fewer than 3 points = empty.
// ------------------------------------------------------------------------------------------
#define NLFEM_MAXSQ 8

__device__ __forceinline__ int nl_sh_pass(const double2* in, int n, int a, double s, double delta, double2* out) {
    if (n == 0) return 0;
    int m = 0;
    double2 S = in[n - 1];
    double sa = a ? S.y : S.x;
    bool s_in = __dmul_rn(s, sa) <= delta;
    for (int i = 0; i < n; ++i) {
        const double2 E = in[i];
        const double ea = a ? E.y : E.x;
        const bool e_in = __dmul_rn(s, ea) <= delta;
        if (e_in != s_in) {
            const double sb = a ? S.x : S.y, eb = a ? E.x : E.y;
            const double sd = __dmul_rn(s, delta);
            const double t = __ddiv_rn(__dsub_rn(sd, sa), __dsub_rn(ea, sa));
            const double xb = __dadd_rn(sb, __dmul_rn(t, __dsub_rn(eb, sb)));
            if (m < NLFEM_MAXSQ) out[m] = a ? make_double2(xb, sd) : make_double2(sd, xb);
            ++m;
        }
        if (e_in) {
            if (m < NLFEM_MAXSQ) out[m] = E;
            ++m;
        }
        S = E;
        sa = ea;
        s_in = e_in;
    }
    return m < NLFEM_MAXSQ ? m : NLFEM_MAXSQ;  // a triangle by four half-planes: at most 7
}

// Polygon of the square cut in coordinates relative to c (rel, up to NLFEM_MAXSQ points);
// returns the point count (0 when empty, 3 with full = true for the whole element).
__device__ __forceinline__ int nl_clip_square_rel(const double2 V[3], double2 c, double delta, double2* rel,
                                                  bool& full) {
    double2 A[NLFEM_MAXSQ], B[NLFEM_MAXSQ];
    bool all_in = true;
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        A[v] = make_double2(__dsub_rn(V[v].x, c.x), __dsub_rn(V[v].y, c.y));
        all_in &= fabs(A[v].x) <= delta && fabs(A[v].y) <= delta;
    }
    full = all_in;
    if (all_in) {
        for (int v = 0; v < 3; ++v) rel[v] = A[v];
        return 3;
    }
    int n = nl_sh_pass(A, 3, 0, 1.0, delta, B);
    n = nl_sh_pass(B, n, 1, 1.0, delta, A);
    n = nl_sh_pass(A, n, 0, -1.0, delta, B);
    n = nl_sh_pass(B, n, 1, -1.0, delta, A);
    int m = 0;
    for (int i = 0; i < n; ++i) {
        if (m > 0 && A[i].x == rel[m - 1].x && A[i].y == rel[m - 1].y) continue;
        rel[m++] = A[i];
    }
    while (m >= 2 && rel[m - 1].x == rel[0].x && rel[m - 1].y == rel[0].y) --m;
    return m >= 3 ? m : 0;
}

// The same cut as CPt points (absolute coordinates c + p, barycentric coordinates in E_l);
// out == nullptr: count only.
__device__ __forceinline__ int nl_clip_square(const double2 V[3], double2 c, double delta, CPt* out, bool& full) {
    double2 rel[NLFEM_MAXSQ];
    const int n = nl_clip_square_rel(V, c, delta, rel, full);
    if (!out || full) return n;
    const double ex1 = V[1].x - V[0].x, ey1 = V[1].y - V[0].y, ex2 = V[2].x - V[0].x, ey2 = V[2].y - V[0].y;
    const double dj = ex1 * ey2 - ey1 * ex2;
    for (int i = 0; i < n; ++i) {
        const double x = __dadd_rn(c.x, rel[i].x), y = __dadd_rn(c.y, rel[i].y);
        const double px = x - V[0].x, py = y - V[0].y;
        out[i] = CPt{x, y, (px * ey2 - py * ex2) / dj, (ex1 * py - ey1 * px) / dj, -1, 0.0, 0};
    }
    return n;
}

// Dispatch on the ball: Euclidean approximations (nocaps / approxcaps) or the infinity ball.
__device__ __forceinline__ int nl_clip_ball(int ball, const double2 V[3], double2 c, double delta, double delta2,
                                            CPt* out, bool& full) {
    if (ball == NLFEM_BALL_INFINITY) return nl_clip_square(V, c, delta, out, full);
    return nl_clip(V, c, delta, delta2, ball == NLFEM_BALL_APPROXCAPS, out, full);
}

// ------------------------------------------------------------------------------------------
// FP32 geometry with exact decisions (bulk quadrature and the pair-search predicate)
//
// R[m] = vertex m of E_l relative to x_p in FP32, C[m] = |R[m]|^2 - delta^2. eps bounds the
// absolute FP32 error of the R components. Each decision the canonical FP64 clip takes is
// taken here only if its margin exceeds a first-order error bound:
//   vertex in ball:    |C| > floor2 + 2 |R|_1 eps
//   chord (both ends outside): |B^2 - A C| > bound(A, B, C, eps)
// nl_decide32 returns false when some decision is too close to call (the caller then uses
// the canonical FP64 clip). Otherwise g holds, per edge, the number of crossings and their
// parameters (increasing); no root snaps or point merges can occur in that case.
// ------------------------------------------------------------------------------------------
struct Geo32 {
    float ta[3], tb[3];
    int nc[3];
    bool in[3];
};

__device__ __forceinline__ bool nl_decide32(const float Rx[3], const float Ry[3], const float C[3], float eps,
                                            float floor2, float d2, Geo32& g) {
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        if (fabsf(C[m]) <= floor2 + 2.f * (fabsf(Rx[m]) + fabsf(Ry[m])) * eps) return false;
        g.in[m] = C[m] < 0.f;
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int b = (e + 1) % 3;
        g.nc[e] = 0;
        g.ta[e] = g.tb[e] = 0.f;
        if (g.in[e] && g.in[b]) continue;
        const float ux = Rx[b] - Rx[e], uy = Ry[b] - Ry[e];
        const float Aq = ux * ux + uy * uy;
        const float Bq = Rx[e] * ux + Ry[e] * uy;
        const float Cq = C[e];
        const float disc = Bq * Bq - Aq * Cq;
        if (g.in[e] != g.in[b]) {
            // exactly one crossing; stable roots, take the one in (0,1)
            const float sq = sqrtf(fmaxf(disc, 0.f));
            const float qq = -(Bq + copysignf(sq, Bq));
            const float r1 = qq / Aq, r2 = Cq / qq;
            g.ta[e] = g.in[e] ? fmaxf(r1, r2) : fminf(r1, r2);
            g.nc[e] = 1;
        } else {
            const float e1n = fabsf(Rx[e]) + fabsf(Ry[e]), u1n = fabsf(ux) + fabsf(uy);
            const float bound = 2.f * fabsf(Bq) * (u1n + 2.f * e1n) * eps + Aq * (2.f * e1n * eps + 1e-6f * d2) +
                                fabsf(Cq) * 4.f * u1n * eps + 1e-6f * (Bq * Bq + fabsf(Aq * Cq));
            if (fabsf(disc) <= bound) return false;
            if (disc > 0.f) {
                const float tc = -Bq / Aq;
                if (tc > 0.f && tc < 1.f) {
                    const float sq = sqrtf(disc);
                    const float qq = -(Bq + copysignf(sq, Bq));
                    const float r1 = qq / Aq, r2 = Cq / qq;
                    g.ta[e] = fminf(r1, r2);
                    g.tb[e] = fmaxf(r1, r2);
                    g.nc[e] = 2;
                }
            }
        }
    }
    return true;
}

// Number of polygon points of a decided configuration (vertices inside, crossings, and
// with caps one cap per consecutive pair not joined along one edge).
__device__ __forceinline__ int nl_count32(const Geo32& g, bool caps) {
    if (g.in[0] && g.in[1] && g.in[2]) return 3;
    int nraw = 0, ncap = 0;
    int fe = 0, fv = 0, le = 0;  // first / last raw point: edge and vertex flag
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int cnt = (g.in[e] ? 1 : 0) + g.nc[e];
        for (int j = 0; j < cnt; ++j) {
            const int v = (j == 0 && g.in[e]) ? 1 : 0;
            // consecutive points on the same edge are joined; else Q must be the next edge's vertex
            if (nraw > 0 && le != e && !(v && e == (le + 1) % 3)) ++ncap;
            if (nraw == 0) { fe = e; fv = v; }
            le = e;
            ++nraw;
        }
    }
    // wrap-around last -> first: joined only if first is the vertex that starts the edge after
    // last's (on one edge the first point never has the larger parameter)
    if (nraw >= 2 && !(fv && fe == (le + 1) % 3)) ++ncap;
    return nraw + (caps && nraw >= 2 ? ncap : 0);
}
