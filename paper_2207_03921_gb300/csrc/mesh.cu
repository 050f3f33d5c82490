// Mesh preparation (Sec. 2.2): counter-clockwise triangles, |det J|, element and node
// labels, node -> element adjacency, centroids and radii for the grid search.
// Also the generic device utilities (scan, segmented sort) the other units use.
#include <algorithm>
#include <climits>

#include "nlfem_internal.cuh"

namespace nlfem {

double elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return (double)ms;
}

// ------------------------------------------------------------------------------------------
// exclusive scan (int64): block scan + recursive scan of block sums
// ------------------------------------------------------------------------------------------
static constexpr int SCAN_B = 1024;

__global__ void k_scan_block(const int64_t* in, int64_t* out, int64_t* bsum, int64_t n) {
    __shared__ int64_t sh[SCAN_B];
    int64_t i = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
    int64_t v = (i < n) ? in[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < SCAN_B; off <<= 1) {
        int64_t t = (threadIdx.x >= (unsigned)off) ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = sh[threadIdx.x] - v;  // exclusive
    if (threadIdx.x == SCAN_B - 1) bsum[blockIdx.x] = sh[threadIdx.x];
}

__global__ void k_scan_add(int64_t* out, const int64_t* boff, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
    if (i < n) out[i] += boff[blockIdx.x];
}

__global__ void k_scan_total(const int64_t* in, const int64_t* ex, int64_t* out_last, int64_t n) {
    *out_last = (n > 0) ? ex[n - 1] + in[n - 1] : 0;
}

static void scan_rec(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    int64_t nb = (n + SCAN_B - 1) / SCAN_B;
    DBuf<int64_t> bsum, boff;
    bsum.alloc(nb, st);
    boff.alloc(nb, st);
    k_scan_block<<<(unsigned)nb, SCAN_B, 0, st>>>(in, out, bsum.p, n);
    NLFEM_LAUNCH_CHECK();
    if (nb > 1) {
        scan_rec(bsum.p, boff.p, nb, st);
        k_scan_add<<<(unsigned)nb, SCAN_B, 0, st>>>(out, boff.p, n);
        NLFEM_LAUNCH_CHECK();
    }
}

// out has n + 1 entries; out[n] = total
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st) {
    if (n > 0) {
        scan_rec(in, out, n, st);
        k_scan_total<<<1, 1, 0, st>>>(in, out, out + n, n);
        NLFEM_LAUNCH_CHECK();
    } else {
        NLFEM_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), st));
    }
}

// ------------------------------------------------------------------------------------------
// segmented sort: one block per segment, bitonic sort in shared memory
// ------------------------------------------------------------------------------------------
template <bool WITH_VALS>
__global__ void k_segsort(int* keys, int* vals, const int64_t* ptr, int cap) {
    extern __shared__ int smem[];
    int* sk = smem;
    int* sv = smem + cap;
    int64_t b = ptr[blockIdx.x], e = ptr[blockIdx.x + 1];
    int len = (int)(e - b);
    if (len <= 1) return;
    int n2 = 1;
    while (n2 < len) n2 <<= 1;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        sk[i] = i < len ? keys[b + i] : INT_MAX;
        if (WITH_VALS) sv[i] = i < len ? vals[b + i] : 0;
    }
    __syncthreads();
    for (int size = 2; size <= n2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                int j = i ^ stride;
                if (j > i) {
                    bool up = (i & size) == 0;
                    int ki = sk[i], kj = sk[j];
                    if ((ki > kj) == up) {
                        sk[i] = kj;
                        sk[j] = ki;
                        if (WITH_VALS) {
                            int t = sv[i];
                            sv[i] = sv[j];
                            sv[j] = t;
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        keys[b + i] = sk[i];
        if (WITH_VALS) vals[b + i] = sv[i];
    }
}

// Short segments (up to 32 * NPL keys): one warp per segment, bitonic network in registers.
// Element e of the padded segment sits in lane e % 32, register e / 32; compare-exchanges
// at strides below 32 go through shuffles, the others stay inside a lane.
template <bool WITH_VALS, int NPL>
__global__ void __launch_bounds__(256) k_segsort_warp(int* keys, int* vals, const int64_t* ptr, int64_t nseg) {
    const int64_t sg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (sg >= nseg) return;  // whole warps
    const int64_t b = ptr[sg];
    const int len = (int)(ptr[sg + 1] - b);
    if (len <= 1) return;
    int v[NPL], w[NPL];
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int e = i * 32 + lane;
        v[i] = e < len ? keys[b + e] : INT_MAX;
        if (WITH_VALS) w[i] = e < len ? vals[b + e] : 0;
    }
#pragma unroll
    for (int size = 2; size <= 32 * NPL; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 32) {
                const int s = stride >> 5;
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    if (i & s) continue;
                    const int j = i | s;
                    const bool up = ((i * 32 + lane) & size) == 0;
                    if ((v[i] > v[j]) == up) {
                        const int t = v[i]; v[i] = v[j]; v[j] = t;
                        if (WITH_VALS) { const int u = w[i]; w[i] = w[j]; w[j] = u; }
                    }
                }
            } else {
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    const int e = i * 32 + lane;
                    const int pv = __shfl_xor_sync(0xffffffffu, v[i], stride);
                    const int pw = WITH_VALS ? __shfl_xor_sync(0xffffffffu, w[i], stride) : 0;
                    const bool up = (e & size) == 0, lower = (e & stride) == 0;
                    // the lower element keeps the smaller key on an ascending run; ties keep the
                    // lower element's own pair so that equal keys never duplicate a value
                    const bool take = lower == up ? (pv < v[i]) : (pv > v[i]);
                    if (take) {
                        v[i] = pv;
                        if (WITH_VALS) w[i] = pw;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int e = i * 32 + lane;
        if (e < len) {
            keys[b + e] = v[i];
            if (WITH_VALS) vals[b + e] = w[i];
        }
    }
}

template <bool WITH_VALS>
static void segsort_warp(int* keys, int* vals, const int64_t* ptr, int64_t nseg, int max_len, cudaStream_t st) {
    const unsigned grid = (unsigned)((nseg * 32 + 255) / 256);
    if (max_len <= 32) k_segsort_warp<WITH_VALS, 1><<<grid, 256, 0, st>>>(keys, vals, ptr, nseg);
    else if (max_len <= 64) k_segsort_warp<WITH_VALS, 2><<<grid, 256, 0, st>>>(keys, vals, ptr, nseg);
    else if (max_len <= 128) k_segsort_warp<WITH_VALS, 4><<<grid, 256, 0, st>>>(keys, vals, ptr, nseg);
    else if (max_len <= 256) k_segsort_warp<WITH_VALS, 8><<<grid, 256, 0, st>>>(keys, vals, ptr, nseg);
    else k_segsort_warp<WITH_VALS, 16><<<grid, 256, 0, st>>>(keys, vals, ptr, nseg);
    NLFEM_LAUNCH_CHECK();
}

void segmented_sort_i32(int* keys, int* vals, const int64_t* ptr, int64_t nseg, int max_len,
                        cudaStream_t st) {
    if (nseg <= 0 || max_len <= 1) return;
    if (max_len <= 512) {  // every segment fits one warp's registers
        if (vals) segsort_warp<true>(keys, vals, ptr, nseg, max_len, st);
        else segsort_warp<false>(keys, nullptr, ptr, nseg, max_len, st);
        return;
    }
    // the whole segment sits in shared memory: 128 KB of keys (and values)
    const int limit = vals ? 16384 : 32768;
    NLFEM_CHECK(max_len <= limit, NLFEM_ERR_UNSUPPORTED,
                "segment of " + std::to_string(max_len) + " entries exceeds the sort capacity " +
                    std::to_string(limit));
    int cap = 1;
    while (cap < max_len) cap <<= 1;
    size_t smem = (size_t)cap * sizeof(int) * (vals ? 2 : 1);
    int threads = std::min(cap / 2 < 32 ? 32 : cap / 2, 512);
    if (vals) {
        NLFEM_CUDA_TRY(cudaFuncSetAttribute(k_segsort<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_segsort<true><<<(unsigned)nseg, threads, smem, st>>>(keys, vals, ptr, cap);
    } else {
        NLFEM_CUDA_TRY(cudaFuncSetAttribute(k_segsort<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_segsort<false><<<(unsigned)nseg, threads, smem, st>>>(keys, nullptr, ptr, cap);
    }
    NLFEM_LAUNCH_CHECK();
}

// ------------------------------------------------------------------------------------------
// mesh kernels
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void atomic_max_d(double* a, double v) {
    unsigned long long* p = (unsigned long long*)a;
    unsigned long long old = *p, assumed;
    while (__longlong_as_double(old) < v) {
        assumed = old;
        old = atomicCAS(p, assumed, __double_as_longlong(v));
        if (old == assumed) break;
    }
}
__device__ __forceinline__ void atomic_min_d(double* a, double v) {
    unsigned long long* p = (unsigned long long*)a;
    unsigned long long old = *p, assumed;
    while (__longlong_as_double(old) > v) {
        assumed = old;
        old = atomicCAS(p, assumed, __double_as_longlong(v));
        if (old == assumed) break;
    }
}

// Orient counter-clockwise exactly as the FP64 determinant's sign says; store |det J|.
__global__ void k_prepare_elems(const int* T3, int64_t K, int64_t M, const double2* X, int4* T,
                                double* det, double2* cen, double* rad, int* err, double* stats,
                                float4* E32, float* det32, ElemRec* rec) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    int t0 = T3[3 * k], t1 = T3[3 * k + 1], t2 = T3[3 * k + 2];
    if (t0 < 0 || t1 < 0 || t2 < 0 || t0 >= M || t1 >= M || t2 >= M) {
        atomicOr(err, 1);
        T[k] = make_int4(0, 0, 0, 0);
        det[k] = 0.0;
        E32[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        det32[k] = 0.f;
        rec[k] = ElemRec{make_double2(0, 0), make_float4(0.f, 0.f, 0.f, 0.f), 0, 0, 0, 0.f};
        return;
    }
    double2 a = X[t0], b = X[t1], c = X[t2];
    double d = __dsub_rn(__dmul_rn(__dsub_rn(b.x, a.x), __dsub_rn(c.y, a.y)),
                         __dmul_rn(__dsub_rn(b.y, a.y), __dsub_rn(c.x, a.x)));
    if (d < 0) {
        int tt = t1; t1 = t2; t2 = tt;
        double2 cc = b; b = c; c = cc;
        d = -d;
    }
    if (!(d > 0)) atomicOr(err, 2);
    T[k] = make_int4(t0, t1, t2, 0);
    det[k] = d;
    E32[k] = make_float4((float)(b.x - a.x), (float)(b.y - a.y), (float)(c.x - a.x), (float)(c.y - a.y));
    det32[k] = (float)d;
    rec[k] = ElemRec{a, E32[k], t0, t1, t2, (float)d};
    double2 ce = make_double2((a.x + b.x + c.x) / 3.0, (a.y + b.y + c.y) / 3.0);
    cen[k] = ce;
    double r = sqrt(fmax(fmax((a.x - ce.x) * (a.x - ce.x) + (a.y - ce.y) * (a.y - ce.y),
                              (b.x - ce.x) * (b.x - ce.x) + (b.y - ce.y) * (b.y - ce.y)),
                         (c.x - ce.x) * (c.x - ce.x) + (c.y - ce.y) * (c.y - ce.y)));
    rad[k] = r;
    atomic_max_d(&stats[0], r);
}

__global__ void k_bbox(const double2* X, int64_t M, double* stats) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    double2 v = X[i];
    atomic_min_d(&stats[1], v.x);
    atomic_min_d(&stats[2], v.y);
    atomic_max_d(&stats[3], v.x);
    atomic_max_d(&stats[4], v.y);
}

__global__ void k_labels(const int8_t* lab_in, int64_t K, int8_t* lab, const int4* T, int8_t* dir) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    int8_t L = lab_in ? (lab_in[k] != 0) : 1;
    lab[k] = L;
    if (!L) {
        int4 t = T[k];
        dir[t.x] = 1;
        dir[t.y] = 1;
        dir[t.z] = 1;
    }
}

__global__ void k_count_ne(const int4* T, int64_t K, int64_t* cnt) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    int4 t = T[k];
    atomicAdd((unsigned long long*)&cnt[t.x], 1ull);
    atomicAdd((unsigned long long*)&cnt[t.y], 1ull);
    atomicAdd((unsigned long long*)&cnt[t.z], 1ull);
}

__global__ void k_fill_ne(const int4* T, int64_t K, const int64_t* ptr, int* cursor, int* idx) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    int4 t = T[k];
    int v[3] = {t.x, t.y, t.z};
    for (int a = 0; a < 3; ++a) {
        int pos = atomicAdd(&cursor[v[a]], 1);
        idx[ptr[v[a]] + pos] = (int)k;
    }
}

__global__ void k_i64_to_i32(const int64_t* a, int* b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (int)a[i];
}

__global__ void k_max_seg(const int64_t* ptr, int64_t n, int* out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    warp_atomic_max(out, i < n ? (int)(ptr[i + 1] - ptr[i]) : 0);
}

int64_t Mesh::device_bytes() const {
    int64_t b = X.bytes() + T.bytes() + det.bytes() + lab.bytes() + dir.bytes() + ne_ptr.bytes() +
                ne_idx.bytes() + cen.bytes() + rad.bytes() + E32.bytes() + det32.bytes() + rec.bytes() +
                Tpos.bytes() + mat.bytes();
    if (cache) {
        const PairCache& c = *cache;
        b += c.pair_ptr.bytes() + c.pk.bytes() + c.pl.bytes() + c.pcls.bytes() + c.pT_ptr.bytes() +
             c.pT_id.bytes() + c.duffy_ids.bytes() + c.nrow_ptr.bytes() + c.ncol.bytes() +
             c.row_ptr.bytes() + c.col.bytes() + c.tpos.bytes() + c.seg_ptr.bytes() + c.idx.bytes() +
             c.pbase.bytes() + c.up_pos.bytes() + c.up_row.bytes() + c.whole_ids.bytes() + c.cut_ids.bytes() +
             c.up_start.bytes() + c.epos.bytes() + c.klr_whole.bytes() + c.klr_cut.bytes() +
             c.kl_whole.bytes();
    }
    return b;
}

static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

__global__ void k_orphans(const int64_t* cnt, int64_t M, int8_t* dir) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M && cnt[i] == 0) dir[i] = 1;  // a node of no element keeps its Dirichlet value
}

// Upload done by the caller: m.X holds the vertices; T3_dev the raw triangles.
// discontinuous ansatz: node 3k + a is a copy of vertex a of element k (as given)
__global__ void k_dg_copy(const double2* X, const int* T3, int64_t K, int64_t M, double2* Xd, int* Td, int* orig,
                          int* err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * K) return;
    int v = T3[i];
    if (v < 0 || v >= M) {
        atomicOr(err, 1);
        v = 0;
    }
    Xd[i] = X[v];
    Td[i] = (int)i;
    orig[i] = v;
}

// position triples of the (oriented) elements: the original vertex of every copy
__global__ void k_dg_tpos(const int4* T, const int* orig, int64_t K, int4* Tpos) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int4 t = T[k];
    Tpos[k] = make_int4(orig[t.x], orig[t.y], orig[t.z], 0);
}

void mesh_make_dg(Mesh& m, const double2* X_dev, int64_t M_in, const int* T3_dev, const int8_t* lab_dev,
                  cudaStream_t st) {
    const int64_t K = m.K;
    m.M = 3 * K;
    m.dg = true;
    m.X.alloc(3 * K, st);
    DBuf<int> Td, orig, err;
    Td.alloc(3 * K, st);
    orig.alloc(3 * K, st);
    err.alloc(1, st);
    err.zero(st);
    k_dg_copy<<<nblk(3 * K, 256), 256, 0, st>>>(X_dev, T3_dev, K, M_in, m.X.p, Td.p, orig.p, err.p);
    NLFEM_LAUNCH_CHECK();
    int herr = 0;
    NLFEM_CUDA_TRY(cudaMemcpyAsync(&herr, err.p, sizeof herr, cudaMemcpyDeviceToHost, st));
    NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
    NLFEM_CHECK(!herr, NLFEM_ERR_BAD_MESH, "triangle vertex index out of range");
    mesh_prepare(m, Td.p, lab_dev, st);
    m.Tpos.alloc(K, st);
    k_dg_tpos<<<nblk(K, 256), 256, 0, st>>>(m.T.p, orig.p, K, m.Tpos.p);
    NLFEM_LAUNCH_CHECK();
    NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
}

void mesh_prepare(Mesh& m, const int* T3_dev, const int8_t* lab_dev, cudaStream_t st) {
    const int64_t K = m.K, M = m.M;
    m.T.alloc(K, st);
    m.det.alloc(K, st);
    m.cen.alloc(K, st);
    m.rad.alloc(K, st);
    m.E32.alloc(K, st);
    m.det32.alloc(K, st);
    m.rec.alloc(K, st);
    m.lab.alloc(K, st);
    m.dir.alloc(M, st);
    m.dir.zero(st);
    DBuf<int> err;
    err.alloc(1, st);
    err.zero(st);
    DBuf<double> stats;
    stats.alloc(5, st);
    double init[5] = {0.0, 1e300, 1e300, -1e300, -1e300};
    NLFEM_CUDA_TRY(cudaMemcpyAsync(stats.p, init, sizeof init, cudaMemcpyHostToDevice, st));
    k_prepare_elems<<<nblk(K, 256), 256, 0, st>>>(T3_dev, K, M, m.X.p, m.T.p, m.det.p, m.cen.p, m.rad.p,
                                                  err.p, stats.p, m.E32.p, m.det32.p, m.rec.p);
    NLFEM_LAUNCH_CHECK();
    k_bbox<<<nblk(M, 256), 256, 0, st>>>(m.X.p, M, stats.p);
    NLFEM_LAUNCH_CHECK();
    int herr = 0;
    double hs[5];
    NLFEM_CUDA_TRY(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    NLFEM_CUDA_TRY(cudaMemcpyAsync(hs, stats.p, sizeof hs, cudaMemcpyDeviceToHost, st));
    NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
    NLFEM_CHECK(!(herr & 1), NLFEM_ERR_BAD_MESH, "triangle vertex index out of range");
    NLFEM_CHECK(!(herr & 2), NLFEM_ERR_BAD_MESH, "triangle with zero area");
    m.rmax = hs[0];
    m.bbox[0] = hs[1];
    m.bbox[1] = hs[2];
    m.bbox[2] = hs[3];
    m.bbox[3] = hs[4];
    k_labels<<<nblk(K, 256), 256, 0, st>>>(lab_dev, K, m.lab.p, m.T.p, m.dir.p);
    NLFEM_LAUNCH_CHECK();
    // node -> elements
    DBuf<int64_t> cnt, ptr;
    cnt.alloc(M, st);
    cnt.zero(st);
    ptr.alloc(M + 1, st);
    k_count_ne<<<nblk(K, 256), 256, 0, st>>>(m.T.p, K, cnt.p);
    NLFEM_LAUNCH_CHECK();
    exclusive_scan_i64(cnt.p, ptr.p, M, st);
    k_orphans<<<nblk(M, 256), 256, 0, st>>>(cnt.p, M, m.dir.p);
    NLFEM_LAUNCH_CHECK();
    m.ne_ptr.alloc(M + 1, st);
    k_i64_to_i32<<<nblk(M + 1, 256), 256, 0, st>>>(ptr.p, m.ne_ptr.p, M + 1);
    NLFEM_LAUNCH_CHECK();
    m.ne_idx.alloc(3 * K, st);
    DBuf<int> cursor;
    cursor.alloc(M, st);
    cursor.zero(st);
    k_fill_ne<<<nblk(K, 256), 256, 0, st>>>(m.T.p, K, ptr.p, cursor.p, m.ne_idx.p);
    NLFEM_LAUNCH_CHECK();
    DBuf<int> mx;
    mx.alloc(1, st);
    mx.zero(st);
    k_max_seg<<<nblk(M, 256), 256, 0, st>>>(ptr.p, M, mx.p);
    NLFEM_LAUNCH_CHECK();
    int hmx = 0;
    NLFEM_CUDA_TRY(cudaMemcpyAsync(&hmx, mx.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
    NLFEM_CHECK(hmx <= 32, NLFEM_ERR_UNSUPPORTED, "a node belongs to more than 32 triangles");
    segmented_sort_i32(m.ne_idx.p, nullptr, ptr.p, M, hmx, st);
}
}  // namespace nlfem
