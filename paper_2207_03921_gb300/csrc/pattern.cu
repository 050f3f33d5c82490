// CSR pattern, slot index and deterministic segmented reduction.
//
// The paper avoids write conflicts on the CPU with one sub-matrix per thread that are
// summed at the end (Sec. 3.4). Here every ordered pair writes its local block on its
// union vertices (pair-major, upper triangle) and a slot index, built once per mesh,
// lists for every upper CSR entry the contributions that belong to it in a fixed order.
// The reduction sums each list in that order and writes the value to both (i,j) and
// (j,i), so A is symmetric to the last bit and identical from run to run.
//
// Contributions of one pair: entry E(a,b), 0 <= a <= b < 6, of the union block
// (union = vertices of E_k, then the vertices of E_l not in E_k). Scalar: 21 values per
// pair; peridynamics: 4 components (c1, c2) per entry, 84 values per pair. Records are
// padded to 24 / 88 values so that no two pairs share a 32-byte sector.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "nlfem_internal.cuh"

namespace nlfem {

static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

__device__ __constant__ int c_E1[6][6] = {
    {0, 1, 2, 3, 4, 5}, {1, 6, 7, 8, 9, 10}, {2, 7, 11, 12, 13, 14},
    {3, 8, 12, 15, 16, 17}, {4, 9, 13, 16, 18, 19}, {5, 10, 14, 17, 19, 20}};

int64_t contrib_entries(int ndof) { return ndof == 1 ? NLFEM_REC1 : NLFEM_REC2; }

static constexpr int MAX_NE = 32;  // elements per node handled by the row enumeration

struct RowEnum {
    const int* ne_ptr;
    const int* ne_idx;
    const int64_t* pair_ptr;
    const int64_t* pT_ptr;
    const int* pT_id;
    const int* pk;
    const int* pl;
    const int4* T;
};

// Per-warp description of node i's contributing pairs: for e in ne(i): the pairs
// (e, *) (x side), then for e in ne(i): the pairs (*, e) whose outer element does not
// contain i (y side). cum[s] = first flattened index of range s.
struct RowRanges {
    int nne;
    int ne[MAX_NE];
    int64_t cum[2 * MAX_NE + 1];
};

__device__ __forceinline__ void row_ranges(const RowEnum& R, int i, RowRanges& rr) {
    int b = R.ne_ptr[i], e = R.ne_ptr[i + 1];
    rr.nne = min(e - b, MAX_NE);
    for (int t = 0; t < rr.nne; ++t) rr.ne[t] = R.ne_idx[b + t];
    rr.cum[0] = 0;
    for (int t = 0; t < rr.nne; ++t)
        rr.cum[t + 1] = rr.cum[t] + (R.pair_ptr[rr.ne[t] + 1] - R.pair_ptr[rr.ne[t]]);
    for (int t = 0; t < rr.nne; ++t)
        rr.cum[rr.nne + t + 1] = rr.cum[rr.nne + t] + (R.pT_ptr[rr.ne[t] + 1] - R.pT_ptr[rr.ne[t]]);
}

// pair id of flattened index f, or -1 if the pair is a y-side duplicate
__device__ __forceinline__ int row_pair(const RowEnum& R, const RowRanges& rr, int64_t f, int i) {
    int s = 0;
    while (rr.cum[s + 1] <= f) ++s;
    int64_t off = f - rr.cum[s];
    if (s < rr.nne) return (int)(R.pair_ptr[rr.ne[s]] + off);
    int e = rr.ne[s - rr.nne];
    int p = R.pT_id[R.pT_ptr[e] + off];
    int4 tk = R.T[R.pk[p]];
    if (tk.x == i || tk.y == i || tk.z == i) return -1;  // already on the x side
    return p;
}

// union vertices of pair p and the position of node i in it
__device__ __forceinline__ int pair_union(const RowEnum& R, int p, int i, int u[6], int& ai) {
    int4 tk = R.T[R.pk[p]], tl = R.T[R.pl[p]];
    u[0] = tk.x; u[1] = tk.y; u[2] = tk.z;
    int U = 3;
    int lv[3] = {tl.x, tl.y, tl.z};
    for (int b = 0; b < 3; ++b) {
        if (lv[b] != u[0] && lv[b] != u[1] && lv[b] != u[2]) u[U++] = lv[b];
    }
    ai = -1;
    for (int a = 0; a < U; ++a)
        if (u[a] == i) ai = a;
    return U;
}

// ------------------------------------------------------------------------------------------
// pattern: per node row, the union vertices of every pair containing the node
// ------------------------------------------------------------------------------------------
// Most inserts repeat a key already present (a node is shared by many pairs of the row), so
// the slot is read first and the compare-and-swap is only issued on an empty slot.
__device__ __forceinline__ bool hash_insert(int* tab, int cap, int key, int* count) {
    unsigned h = ((unsigned)key * 2654435761u) & (unsigned)(cap - 1);
    for (int probe = 0; probe < cap; ++probe) {
        int cur = tab[h];
        if (cur == key) return true;
        if (cur == -1) {
            cur = atomicCAS(&tab[h], -1, key);
            if (cur == -1) {
                atomicAdd(count, 1);
                return true;
            }
            if (cur == key) return true;
        }
        h = (h + 1) & (unsigned)(cap - 1);
    }
    return false;
}

// the row's keys gathered from the table (in any order), bitonic-sorted over the next power
// of two and written to out
__device__ __forceinline__ void sorted_row(const int* tab, int* keys, int cap, int n, int* out) {
    __shared__ int wpos;
    if (threadIdx.x == 0) wpos = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < cap; t += blockDim.x) {
        const int key = tab[t];
        if (key != -1) keys[atomicAdd(&wpos, 1)] = key;
    }
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    __syncthreads();
    for (int t = n + threadIdx.x; t < n2; t += blockDim.x) keys[t] = 0x7fffffff;
    __syncthreads();
    for (int size = 2; size <= n2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < n2; t += blockDim.x) {
                const int j = t ^ stride;
                if (j > t) {
                    const bool up = (t & size) == 0;
                    const int a = keys[t], b = keys[j];
                    if ((a > b) == up) {
                        keys[t] = b;
                        keys[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < n; t += blockDim.x) out[t] = keys[t];
}

// One block per node row: its threads share the row's hash table (cap ints) and a buffer
// for the compacted keys (cap / 2 ints). A row visits every pair of its node's elements, tens
// of thousands for wide horizons, through chains of dependent loads; a whole block on one
// row keeps enough of them in flight.
// FILL = false: count the columns of each row; true: write the sorted columns at rowptr[i],
// or with SLOTS at i * cap / 2 and count them (one pass; k_compact_rows packs the slots)
static constexpr int PAT_THREADS = 256;

template <bool FILL, bool SLOTS = false>
__global__ void __launch_bounds__(PAT_THREADS) k_pattern(RowEnum R, int64_t M, int cap, int64_t* rowcnt,
                                                         const int64_t* rowptr, int* cols, int* overflow) {
    extern __shared__ int sm[];
    __shared__ RowRanges rr;
    __shared__ int count, bad;
    const int64_t i = blockIdx.x;
    if (i >= M) return;
    int* tab = sm;
    int* keys = sm + cap;
    for (int t = threadIdx.x; t < cap; t += blockDim.x) tab[t] = -1;
    if (threadIdx.x == 0) {
        row_ranges(R, (int)i, rr);
        count = 0;
        bad = 0;
    }
    __syncthreads();
    const int64_t total = rr.cum[2 * rr.nne];
    bool ok = true;
    // the union vertices of every pair containing i: the nodes of i's own elements once, and
    // per pair the nodes of its other element (E_l on the x side, E_k on the y side)
    for (int t = threadIdx.x; t < rr.nne; t += blockDim.x) {
        const int4 te = R.T[rr.ne[t]];
        ok &= hash_insert(tab, cap, te.x, &count);
        ok &= hash_insert(tab, cap, te.y, &count);
        ok &= hash_insert(tab, cap, te.z, &count);
    }
    int s = 0;  // range of f: a thread's f only grows, so its range index does too
    for (int64_t f = threadIdx.x; f < total; f += blockDim.x) {
        while (rr.cum[s + 1] <= f) ++s;
        const int64_t off = f - rr.cum[s];
        int4 to;
        if (s < rr.nne) {
            to = R.T[R.pl[R.pair_ptr[rr.ne[s]] + off]];
        } else {
            const int e = rr.ne[s - rr.nne];
            const int p = R.pT_id[R.pT_ptr[e] + off];
            to = R.T[R.pk[p]];
            if (to.x == (int)i || to.y == (int)i || to.z == (int)i) continue;  // already on the x side
        }
        ok &= hash_insert(tab, cap, to.x, &count);
        ok &= hash_insert(tab, cap, to.y, &count);
        ok &= hash_insert(tab, cap, to.z, &count);
    }
    if (!ok) bad = 1;
    __syncthreads();
    const int n = count;
    if (bad || n > cap / 2) {
        if (threadIdx.x == 0) atomicOr(overflow, 1);
        return;
    }
    if (!FILL || SLOTS) {
        if (threadIdx.x == 0) rowcnt[i] = n;
    }
    if constexpr (FILL) sorted_row(tab, keys, cap, n, cols + (SLOTS ? i * (int64_t)(cap / 2) : rowptr[i]));
}

__global__ void k_compact_rows(const int* slots, int64_t M, int64_t width, const int64_t* ptr, int* out) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= M) return;
    const int64_t b = ptr[i], n = ptr[i + 1] - b;
    for (int64_t j = lane; j < n; j += 32) out[b + j] = slots[i * width + j];
}

// dof-level CSR from the node-level pattern (dofs of a node are interleaved)
__global__ void k_expand_rows(const int64_t* nptr, int64_t M, int ndof, int64_t* row_ptr) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > M) return;
    if (i == M) {
        row_ptr[M * ndof] = (int64_t)ndof * ndof * nptr[M];
        return;
    }
    int64_t n = nptr[i + 1] - nptr[i];
    for (int c = 0; c < ndof; ++c) row_ptr[i * ndof + c] = (int64_t)ndof * ndof * nptr[i] + c * ndof * n;
}

__device__ __forceinline__ int64_t find_col(const int* col, int64_t b, int64_t e, int key) {
    while (b < e) {
        int64_t mid = (b + e) >> 1;
        if (col[mid] < key) b = mid + 1;
        else e = mid;
    }
    return b;
}

// dof columns and the transpose map (thread per node-pattern entry)
__global__ void k_expand_cols(const int64_t* nptr, const int* ncol, int64_t M, int ndof,
                              const int64_t* row_ptr, int* col, int64_t* tpos, int* ntpos, int* err) {
    int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (i >= M) return;
    int64_t b = nptr[i], e = nptr[i + 1];
    for (int64_t t = b + lane; t < e; t += 32) {
        int j = ncol[t];
        int64_t r = t - b;
        int64_t rt = find_col(ncol, nptr[j], nptr[j + 1], (int)i) - nptr[j];  // rank of i in row j
        if (rt >= nptr[j + 1] - nptr[j] || ncol[nptr[j] + rt] != (int)i) {  // the pattern is symmetric
            atomicOr(err, 1);
            rt = 0;
        }
        ntpos[t] = (int)rt;
        for (int c1 = 0; c1 < ndof; ++c1)
            for (int c2 = 0; c2 < ndof; ++c2) {
                int64_t s = row_ptr[i * ndof + c1] + ndof * r + c2;
                col[s] = j * ndof + c2;
                tpos[s] = row_ptr[(int64_t)j * ndof + c2] + ndof * rt + c1;
            }
    }
}

// ------------------------------------------------------------------------------------------
// slot index: for every node-level upper entry (i, j >= i) the list of (pair, entry)
// contributions, in the fixed order of the row enumeration
// ------------------------------------------------------------------------------------------
template <bool FILL>
__global__ void k_slots(RowEnum R, int64_t M, const int64_t* nptr, const int* ncol, int maxrow,
                        int64_t* seg_cnt, const int64_t* seg_ptr, uint64_t* idx, int64_t* pbase,
                        int* overflow) {
    extern __shared__ int sm[];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    int* rcols = sm + warp * 2 * maxrow;
    int* cur = rcols + maxrow;
    if (i >= M) return;
    int64_t rb = nptr[i], re = nptr[i + 1];
    int n = (int)(re - rb);
    for (int t = lane; t < n; t += 32) {
        rcols[t] = ncol[rb + t];
        cur[t] = 0;
    }
    __syncwarp();
    RowRanges rr;
    row_ranges(R, (int)i, rr);
    int64_t total = rr.cum[2 * rr.nne];
    // first pair id the row refers to
    long long pmin = 0x7fffffffffffffffll;
    for (int64_t f0 = 0; f0 < total; f0 += 32) {
        int64_t f = f0 + lane;
        if (f < total) {
            int p = row_pair(R, rr, f, (int)i);
            if (p >= 0) pmin = min(pmin, (long long)p);
        }
    }
    for (int o = 16; o > 0; o >>= 1) pmin = min(pmin, __shfl_xor_sync(0xffffffffu, pmin, o));
    if (!FILL && lane == 0) pbase[i] = pmin;
    int64_t pb = FILL ? pbase[i] : pmin;
    bool bad = false;
    for (int64_t f0 = 0; f0 < total; f0 += 32) {
        int64_t f = f0 + lane;
        int p = -1;
        if (f < total) p = row_pair(R, rr, f, (int)i);
        int u[6] = {0, 0, 0, 0, 0, 0}, ai = 0, U = 0;
        if (p >= 0) U = pair_union(R, p, (int)i, u, ai);
        for (int b = 0; b < 6; ++b) {
            int key = -1;
            if (b < U && u[b] >= (int)i) {
                key = (int)(find_col(rcols, 0, n, u[b]));
                if (key >= n || rcols[key] != u[b]) {  // every union vertex is in the row
                    bad = true;
                    key = -1;
                }
            }
            unsigned act = __ballot_sync(0xffffffffu, key >= 0);
            if (!act) continue;
            unsigned grp = __match_any_sync(0xffffffffu, key);
            if (key >= 0) {
                int leader = __ffs(grp) - 1;
                int rank = __popc(grp & ((1u << lane) - 1u));
                if (!FILL) {
                    if (lane == leader) cur[key] += __popc(grp);
                } else {
                    int base = 0;
                    if (lane == leader) {
                        base = cur[key];
                        cur[key] = base + __popc(grp);
                    }
                    base = __shfl_sync(grp, base, leader);
                    int a = ai, bb = b;
                    uint32_t tflag = 0;
                    if (a > bb) {
                        int tt = a; a = bb; bb = tt;
                        tflag = 1;
                    }
                    int64_t rel = (int64_t)p - pb;
                    if (rel < 0) bad = true;
                    idx[seg_ptr[rb + key] + base + rank] =
                        ((uint64_t)rel << 6) | ((uint64_t)tflag << 5) | (uint64_t)c_E1[a][bb];
                }
            }
            __syncwarp();
        }
    }
    if (bad) atomicOr(overflow, 2);  // a pair too far from the row's first pair, or a missing column
    __syncwarp();
    if (!FILL)
        for (int t = lane; t < n; t += 32) seg_cnt[rb + t] = cur[t];
}

// ------------------------------------------------------------------------------------------
// segmented reduction: one warp per node-level upper CSR entry (i, j >= i). Lanes read the
// segment's index entries coalesced and gather the contributions; each lane sums its
// strided share (TwoSum-compensated in FP32 for the bulk path, FP64 for the plain path),
// and the 32 partial sums are combined in a fixed butterfly, so the result is the same on
// every run. The value is written to (i, j) and (j, i).
// ------------------------------------------------------------------------------------------
struct CSum {
    float hi, lo;
};

__device__ __forceinline__ void two_sum_add(CSum& a, float x) {
    float s = a.hi + x;
    float bp = s - a.hi;
    a.lo += (a.hi - (s - bp)) + (x - bp);
    a.hi = s;
}

__device__ __forceinline__ void two_sum_merge(CSum& a, const CSum& b) {
    two_sum_add(a, b.hi);
    a.lo += b.lo;
}

template <typename R>
__device__ __forceinline__ double warp_total(R v);

template <>
__device__ __forceinline__ double warp_total<double>(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_total_c(CSum c) {
    for (int o = 16; o > 0; o >>= 1) {
        CSum d;
        d.hi = __shfl_xor_sync(0xffffffffu, c.hi, o);
        d.lo = __shfl_xor_sync(0xffffffffu, c.lo, o);
        // combine in a lane-independent order so all lanes agree bit for bit
        CSum a = (threadIdx.x & o) ? d : c, b = (threadIdx.x & o) ? c : d;
        two_sum_merge(a, b);
        c = a;
    }
    return (double)c.hi + (double)c.lo;
}

// Half a warp per upper entry (two entries per warp in flight); each lane issues the loads
// of its first four contributions before summing them, so a lane keeps up to eight
// independent loads in flight. The order of the sum is fixed by the slot index.
template <typename R, int NDOF>
__global__ void __launch_bounds__(256) k_reduce(int64_t n_upper, const int64_t* __restrict__ up_pos,
                                                const int* __restrict__ up_row, const int64_t* __restrict__ nptr,
                                                const int* __restrict__ ncol, const int64_t* __restrict__ seg_ptr,
                                                const uint64_t* __restrict__ idx, const int64_t* __restrict__ pbase,
                                                const R* __restrict__ contrib, const int64_t* __restrict__ row_ptr,
                                                const int64_t* __restrict__ tpos, double* __restrict__ val) {
    constexpr int SUB = 16;
    constexpr int NS = NDOF == 1 ? NLFEM_REC1 : NLFEM_REC2;  // record stride
    constexpr int NCOMP = NDOF == 1 ? 1 : 4;
    constexpr int UNR = 4;
    const int sl = threadIdx.x & (SUB - 1);
    const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / SUB;
    const bool live = u < n_upper;  // every lane reaches the shuffles below
    int64_t t = 0, s0 = 0, s1 = 0, pb = 0;
    int i = 0;
    if (live) {
        t = up_pos[u];
        i = up_row[u];
        s0 = seg_ptr[t];
        s1 = seg_ptr[t + 1];
        pb = pbase[i];
    }
    using Acc = typename std::conditional<sizeof(R) == 4, CSum, double>::type;
    Acc acc[NCOMP];
#pragma unroll
    for (int k = 0; k < NCOMP; ++k) {
        if constexpr (sizeof(R) == 4) acc[k] = CSum{0.f, 0.f};
        else acc[k] = 0.0;
    }
    auto load = [&](uint64_t e, R (&x)[NCOMP]) {
        const R* cp = contrib + (pb + (int64_t)(e >> 6)) * NS + (e & 31) * NCOMP;
        if constexpr (NDOF == 1) {
            x[0] = cp[0];
        } else {
            const bool tr = (e >> 5) & 1;  // the entry was stored for (j, i): swap xy and yx
            R y[4];
            if constexpr (sizeof(R) == 4) {
                const float4 f = *reinterpret_cast<const float4*>(cp);
                y[0] = f.x; y[1] = f.y; y[2] = f.z; y[3] = f.w;
            } else {
                y[0] = cp[0]; y[1] = cp[1]; y[2] = cp[2]; y[3] = cp[3];
            }
            x[0] = y[0];
            x[1] = tr ? y[2] : y[1];
            x[2] = tr ? y[1] : y[2];
            x[3] = y[3];
        }
    };
    auto add = [&](const R (&x)[NCOMP]) {
#pragma unroll
        for (int k = 0; k < NCOMP; ++k) {
            if constexpr (sizeof(R) == 4) two_sum_add(acc[k], x[k]);
            else acc[k] += x[k];
        }
    };
    {
        uint64_t e[UNR];
#pragma unroll
        for (int r = 0; r < UNR; ++r) {
            const int64_t q = s0 + sl + (int64_t)SUB * r;
            e[r] = q < s1 ? idx[q] : 0ull;
        }
        R x[UNR][NCOMP];
#pragma unroll
        for (int r = 0; r < UNR; ++r)
            if (s0 + sl + (int64_t)SUB * r < s1) load(e[r], x[r]);
#pragma unroll
        for (int r = 0; r < UNR; ++r)
            if (s0 + sl + (int64_t)SUB * r < s1) add(x[r]);
    }
    for (int64_t q = s0 + sl + (int64_t)SUB * UNR; q < s1; q += SUB) {
        R x[NCOMP];
        load(idx[q], x);
        add(x);
    }
    // fixed butterfly over the half warp; the two operands are combined in a lane-independent
    // order, so all lanes agree to the last bit
    double v[NCOMP];
#pragma unroll
    for (int k = 0; k < NCOMP; ++k) {
        if constexpr (sizeof(R) == 4) {
            CSum c = acc[k];
#pragma unroll
            for (int o = SUB / 2; o > 0; o >>= 1) {
                CSum d;
                d.hi = __shfl_xor_sync(0xffffffffu, c.hi, o);
                d.lo = __shfl_xor_sync(0xffffffffu, c.lo, o);
                CSum a = (sl & o) ? d : c, b = (sl & o) ? c : d;
                two_sum_merge(a, b);
                c = a;
            }
            v[k] = 0.0;
            if (sl == 0) v[k] = (double)c.hi + (double)c.lo;
        } else {
            double a = acc[k];
#pragma unroll
            for (int o = SUB / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            v[k] = a;
        }
    }
    if (!live || sl != 0) return;
    if constexpr (NDOF == 1) {
        const int64_t s = row_ptr[i] + (t - nptr[i]);
        val[s] = v[0];
        val[tpos[s]] = v[0];
    } else {
        const int j = ncol[t];
        const int64_t r = t - nptr[i];
        for (int c1 = 0; c1 < 2; ++c1)
            for (int c2 = 0; c2 < 2; ++c2) {
                if (j == i && c2 < c1) continue;  // the diagonal node block: upper dofs only
                const int64_t s = row_ptr[(int64_t)i * 2 + c1] + 2 * r + c2;
                val[s] = v[c1 * 2 + c2];
                val[tpos[s]] = v[c1 * 2 + c2];
            }
    }
}

// list of node-level upper entries (i, j >= i): pattern position and row
__global__ void k_upper_count(const int64_t* nptr, const int* ncol, int64_t M, int64_t* cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    int64_t b = nptr[i], e = nptr[i + 1];
    int64_t c = 0;
    for (int64_t t = b; t < e; ++t) c += ncol[t] >= (int)i;
    cnt[i] = c;
}

// node rows in strip-sweep order: cells of a uniform grid about one node spacing wide are
// grouped into vertical strips of SW cells, the strips are taken left to right and each is
// swept bottom to top row of cells by row of cells (rows of a cell by node index). The
// entries in flight then lie in a band a few cell rows high inside one strip, and the
// rows of any pair's nodes (at most delta + 2h apart) are reached within a few strip
// widths of rows of each other, so the pair's contributions are re-read from L2.
__global__ void k_node_cell(const double2* X, int64_t M, double x0, double y0, double cs, int nx, int ny, int sw,
                            int64_t* cnt, int* cell) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    double2 v = X[i];
    int cx = min(nx - 1, max(0, (int)floor((v.x - x0) / cs)));
    int cy = min(ny - 1, max(0, (int)floor((v.y - y0) / cs)));
    int c = ((cx / sw) * ny + cy) * sw + (cx % sw);
    cell[i] = c;
    atomicAdd((unsigned long long*)&cnt[c], 1ull);
}

__global__ void k_node_place(const int* cell, int64_t M, const int64_t* start, int* cursor, int* order) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    int pos = atomicAdd(&cursor[cell[i]], 1);
    order[start[cell[i]] + pos] = (int)i;
}

__global__ void k_gather_i64(const int64_t* a, const int* order, int64_t n, int64_t* b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[order[i]];
}

__global__ void k_upper_fill(const int64_t* nptr, const int* ncol, int64_t M, const int64_t* off, int64_t* up_pos,
                             int* up_row, const int* order) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= M) return;
    const int64_t i = order[r];
    int64_t b = nptr[i], e = nptr[i + 1];
    int64_t o = off[r];
    for (int64_t t = b; t < e; ++t)
        if (ncol[t] >= (int)i) {
            up_pos[o] = t;
            up_row[o] = (int)i;
            ++o;
        }
}

__global__ void k_row_max(const int64_t* ptr, int64_t n, int* out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    warp_atomic_max(out, i < n ? (int)(ptr[i + 1] - ptr[i]) : 0);
}

void build_pattern(Mesh& m, PairCache& pc, cudaStream_t st) {
    const int64_t M = m.M;
    RowEnum R{m.ne_ptr.p, m.ne_idx.p, pc.pair_ptr.p, pc.pT_ptr.p, pc.pT_id.p, pc.pk.p, pc.pl.p, m.T.p};
    DBuf<int> ovf;
    ovf.alloc(1, st);
    DBuf<int64_t> rowcnt;
    rowcnt.alloc(M, st);
    pc.nrow_ptr.alloc(M + 1, st);
    // table capacity: twice the node count of a row's pairs is an upper bound on its columns
    // (at most 3 new nodes per partner element); start from the largest partner list
    const int64_t maxp = std::max(max_segment_i64(pc.pair_ptr.p, m.K, st), max_segment_i64(pc.pT_ptr.p, m.K, st));
    int cap = 1024;
    while (cap < 32768 && cap < 2 * maxp) cap *= 2;
    for (;;) {
        ovf.zero(st);
        const size_t smem = (size_t)(cap + cap / 2) * sizeof(int);  // table and compacted keys
        NLFEM_CUDA_TRY(cudaFuncSetAttribute(k_pattern<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        NLFEM_CUDA_TRY(cudaFuncSetAttribute(k_pattern<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        NLFEM_CUDA_TRY(
            cudaFuncSetAttribute(k_pattern<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        // one pass into per-row slots (a row has at most cap / 2 columns) when they fit in 4 GB
        const bool slots = M * (int64_t)(cap / 2) * (int64_t)sizeof(int) <= ((int64_t)4 << 30);
        DBuf<int> slot_buf;
        if (slots) {
            slot_buf.alloc(M * (int64_t)(cap / 2), st);
            k_pattern<true, true><<<(unsigned)M, PAT_THREADS, smem, st>>>(R, M, cap, rowcnt.p, nullptr, slot_buf.p,
                                                                          ovf.p);
        } else {
            k_pattern<false><<<(unsigned)M, PAT_THREADS, smem, st>>>(R, M, cap, rowcnt.p, nullptr, nullptr, ovf.p);
        }
        NLFEM_LAUNCH_CHECK();
        int h = 0;
        NLFEM_CUDA_TRY(cudaMemcpyAsync(&h, ovf.p, sizeof h, cudaMemcpyDeviceToHost, st));
        NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
        if (!h) {
            exclusive_scan_i64(rowcnt.p, pc.nrow_ptr.p, M, st);
            NLFEM_CUDA_TRY(cudaMemcpyAsync(&pc.nnz_node, pc.nrow_ptr.p + M, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
            pc.ncol.alloc(pc.nnz_node, st);
            if (slots) {
                k_compact_rows<<<nblk(M * 32, 256), 256, 0, st>>>(slot_buf.p, M, cap / 2, pc.nrow_ptr.p, pc.ncol.p);
            } else {
                k_pattern<true><<<(unsigned)M, PAT_THREADS, smem, st>>>(R, M, cap, rowcnt.p, pc.nrow_ptr.p,
                                                                        pc.ncol.p, ovf.p);
            }
            NLFEM_LAUNCH_CHECK();
            break;
        }
        cap *= 4;
        NLFEM_CHECK(cap <= 32768, NLFEM_ERR_UNSUPPORTED, "a CSR row would exceed 16384 columns");
    }
    // row length statistics
    {
        DBuf<int> mx;
        mx.alloc(1, st);
        mx.zero(st);
        k_row_max<<<nblk(M, 256), 256, 0, st>>>(pc.nrow_ptr.p, M, mx.p);
        NLFEM_LAUNCH_CHECK();
        NLFEM_CUDA_TRY(cudaMemcpyAsync(&pc.max_row, mx.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
    }
    const int nd = pc.ndof;
    pc.N = M * nd;
    pc.nnz = pc.nnz_node * nd * nd;
    pc.row_ptr.alloc(pc.N + 1, st);
    k_expand_rows<<<nblk(M + 1, 256), 256, 0, st>>>(pc.nrow_ptr.p, M, nd, pc.row_ptr.p);
    NLFEM_LAUNCH_CHECK();
    pc.col.alloc(pc.nnz, st);
    pc.tpos.alloc(pc.nnz, st);
    pc.ntpos.alloc(pc.nnz_node, st);
    ovf.zero(st);
    k_expand_cols<<<nblk(M, 8), 256, 0, st>>>(pc.nrow_ptr.p, pc.ncol.p, M, nd, pc.row_ptr.p, pc.col.p, pc.tpos.p,
                                              pc.ntpos.p, ovf.p);
    NLFEM_LAUNCH_CHECK();
    {
        int h = 0;
        NLFEM_CUDA_TRY(cudaMemcpyAsync(&h, ovf.p, sizeof h, cudaMemcpyDeviceToHost, st));
        NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
        NLFEM_CHECK(!h, NLFEM_ERR_CUDA, "internal error: the CSR pattern is not symmetric");
    }
    // upper entries per row (node order): the numbering of the FP32-bulk accumulators
    {
        DBuf<int64_t> ucnt;
        ucnt.alloc(M, st);
        k_upper_count<<<nblk(M, 256), 256, 0, st>>>(pc.nrow_ptr.p, pc.ncol.p, M, ucnt.p);
        NLFEM_LAUNCH_CHECK();
        pc.up_start.alloc(M + 1, st);
        exclusive_scan_i64(ucnt.p, pc.up_start.p, M, st);
        NLFEM_CUDA_TRY(cudaMemcpyAsync(&pc.n_upper, pc.up_start.p + M, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
    }
    pc.slots_built = false;
}

// Slot index and the ordered list of upper entries of the ordered reduction (FP64 path),
// built on first use.
void build_slots(Mesh& m, PairCache& pc, cudaStream_t st) {
    const int64_t M = m.M;
    RowEnum R{m.ne_ptr.p, m.ne_idx.p, pc.pair_ptr.p, pc.pT_ptr.p, pc.pT_id.p, pc.pk.p, pc.pl.p, m.T.p};
    DBuf<int> ovf;
    ovf.alloc(1, st);
    // slot index
    DBuf<int64_t> segcnt;
    segcnt.alloc(pc.nnz_node, st);
    pc.seg_ptr.alloc(pc.nnz_node + 1, st);
    pc.pbase.alloc(M, st);
    int maxrow = std::max(pc.max_row, 1);
    int warps = std::max(1, std::min(8, (int)(180 * 1024 / (2 * maxrow * 4))));
    size_t smem = (size_t)warps * 2 * maxrow * sizeof(int);
    NLFEM_CHECK(smem <= 200 * 1024, NLFEM_ERR_UNSUPPORTED, "CSR row too long for the slot index");
    NLFEM_CUDA_TRY(cudaFuncSetAttribute(k_slots<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    NLFEM_CUDA_TRY(cudaFuncSetAttribute(k_slots<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    ovf.zero(st);
    k_slots<false><<<nblk(M, warps), warps * 32, smem, st>>>(R, M, pc.nrow_ptr.p, pc.ncol.p, maxrow, segcnt.p,
                                                             nullptr, nullptr, pc.pbase.p, ovf.p);
    NLFEM_LAUNCH_CHECK();
    exclusive_scan_i64(segcnt.p, pc.seg_ptr.p, pc.nnz_node, st);
    NLFEM_CUDA_TRY(cudaMemcpyAsync(&pc.ncontrib, pc.seg_ptr.p + pc.nnz_node, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
    pc.idx.alloc(pc.ncontrib, st);
    k_slots<true><<<nblk(M, warps), warps * 32, smem, st>>>(R, M, pc.nrow_ptr.p, pc.ncol.p, maxrow, nullptr,
                                                            pc.seg_ptr.p, pc.idx.p, pc.pbase.p, ovf.p);
    NLFEM_LAUNCH_CHECK();
    int h = 0;
    NLFEM_CUDA_TRY(cudaMemcpyAsync(&h, ovf.p, sizeof h, cudaMemcpyDeviceToHost, st));
    NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
    NLFEM_CHECK(!(h & 2), NLFEM_ERR_UNSUPPORTED,
                "the slot index misses a column of a CSR row");
    // node-level upper entries, the work items of the reduction, in 2D tile order of the rows
    DBuf<int> order;
    order.alloc(M, st);
    {
        const double W = m.bbox[2] - m.bbox[0], H = m.bbox[3] - m.bbox[1];
        double cs = std::sqrt(std::max(W * H, 1e-300) / (double)M);  // about one node per cell
        if (!(cs > 0)) cs = 1.0;
        int nx = std::max(1, (int)std::ceil(W / cs)), ny = std::max(1, (int)std::ceil(H / cs));
        while ((int64_t)nx * ny > (1 << 22)) {
            cs *= 2.0;
            nx = std::max(1, (int)std::ceil(W / cs));
            ny = std::max(1, (int)std::ceil(H / cs));
        }
        const int sw = std::min(nx, 128);  // strip width in cells
        const int64_t nc = (int64_t)((nx + sw - 1) / sw) * ny * sw;
        DBuf<int64_t> ccnt, cstart;
        DBuf<int> cell, cur;
        ccnt.alloc(nc, st);
        ccnt.zero(st);
        cstart.alloc(nc + 1, st);
        cell.alloc(M, st);
        cur.alloc(nc, st);
        cur.zero(st);
        k_node_cell<<<nblk(M, 256), 256, 0, st>>>(m.X.p, M, m.bbox[0], m.bbox[1], cs, nx, ny, sw, ccnt.p, cell.p);
        NLFEM_LAUNCH_CHECK();
        exclusive_scan_i64(ccnt.p, cstart.p, nc, st);
        k_node_place<<<nblk(M, 256), 256, 0, st>>>(cell.p, M, cstart.p, cur.p, order.p);
        NLFEM_LAUNCH_CHECK();
        DBuf<unsigned long long> mx;
        DBuf<int> mxi;
        mxi.alloc(1, st);
        mxi.zero(st);
        k_row_max<<<nblk(nc, 256), 256, 0, st>>>(cstart.p, nc, mxi.p);
        NLFEM_LAUNCH_CHECK();
        int hm = 0;
        NLFEM_CUDA_TRY(cudaMemcpyAsync(&hm, mxi.p, sizeof hm, cudaMemcpyDeviceToHost, st));
        NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
        segmented_sort_i32(order.p, nullptr, cstart.p, nc, hm, st);  // deterministic order within a tile
    }
    DBuf<int64_t> ucnt, ucnt_o, uoff;
    ucnt.alloc(M, st);
    ucnt_o.alloc(M, st);
    uoff.alloc(M + 1, st);
    k_upper_count<<<nblk(M, 256), 256, 0, st>>>(pc.nrow_ptr.p, pc.ncol.p, M, ucnt.p);
    NLFEM_LAUNCH_CHECK();
    k_gather_i64<<<nblk(M, 256), 256, 0, st>>>(ucnt.p, order.p, M, ucnt_o.p);
    NLFEM_LAUNCH_CHECK();
    exclusive_scan_i64(ucnt_o.p, uoff.p, M, st);
    pc.up_pos.alloc(pc.n_upper, st);
    pc.up_row.alloc(pc.n_upper, st);
    k_upper_fill<<<nblk(M, 256), 256, 0, st>>>(pc.nrow_ptr.p, pc.ncol.p, M, uoff.p, pc.up_pos.p, pc.up_row.p,
                                               order.p);
    NLFEM_LAUNCH_CHECK();
    NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
    pc.slots_built = true;
}

// ------------------------------------------------------------------------------------------
// FP32-bulk accumulation index and the conversion of the fixed-point sums into CSR values
// ------------------------------------------------------------------------------------------
// position of the diagonal within each node row (its first column >= the row)
__global__ void k_diag(const int64_t* __restrict__ nptr, const int* __restrict__ ncol, int64_t M, int* __restrict__ diag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    int64_t a = nptr[i], c = nptr[i + 1];
    while (a < c) {
        const int64_t mid = (a + c) >> 1;
        if (ncol[mid] < (int)i) a = mid + 1;
        else c = mid;
    }
    diag[i] = (int)(a - nptr[i]);
}

__global__ void k_epos(const int4* __restrict__ T, int64_t K, const int64_t* __restrict__ nptr,
                       const int* __restrict__ ncol, const int64_t* __restrict__ up_start, int* __restrict__ epos,
                       int* ovf) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int4 t = T[k];
    const int n[3] = {t.x, t.y, t.z};
    const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {0, 1, 2, 1, 2, 2};
    for (int e = 0; e < 6; ++e) {
        const int i = n[pa[e]], j = n[pb[e]], lo = min(i, j), hi = max(i, j);
        const int r = upper_rank(nptr, ncol, lo, hi);
        if (r < 0) atomicOr(ovf, 1);
        const int64_t u = up_start[lo] + max(r, 0);
        if (u > 0x7fffffffll) atomicOr(ovf, 4);
        epos[k * 8 + e] = (int)u;
    }
    epos[k * 8 + 6] = epos[k * 8 + 7] = 0;
}

// kl ranks of a list: for node pair (x, y) = (vertex a of E_k, vertex b of E_l) the rank of the
// larger node in the upper part of the smaller one's row. Both cases search y in row x, which
// the warp's pairs (most of them with the same E_k) share: rank = position - diag[x] for y >= x,
// and ntpos (the rank of x in row y) - diag[y] for y < x.
__global__ void k_klr(const int* __restrict__ ids, int64_t n, const int* __restrict__ pk, const int* __restrict__ pl,
                      const int4* __restrict__ T, const int64_t* __restrict__ nptr, const int* __restrict__ ncol,
                      const int* __restrict__ ntpos, const int* __restrict__ diag, uint16_t* __restrict__ klr,
                      int* ovf) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = ids[i];
    const int4 a4 = T[pk[p]], b4 = T[pl[p]];
    const int kn[3] = {a4.x, a4.y, a4.z}, ln[3] = {b4.x, b4.y, b4.z};
    for (int a = 0; a < 3; ++a) {
        const int x = kn[a];
        const int64_t rb = nptr[x];
        const int len = (int)(nptr[x + 1] - rb);
        const int* const row = ncol + rb;
        // the largest power of two not above the row length: a branch-free bisection in 32-bit
        // offsets (the kernel is bound by its integer pipe)
        const int top = len > 0 ? 1 << (31 - __clz(len)) : 0;
        for (int b = 0; b < 3; ++b) {
            const int y = ln[b];
            // lower bound of y in row[0, len)
            int lo = 0;
            if (top && row[top - 1] < y) lo = len - top;
            for (int step = top >> 1; step > 0; step >>= 1)
                if (row[lo + step - 1] < y) lo += step;
            if (top && lo < len && row[lo] < y) ++lo;
            int r = -1;
            if (lo < len && row[lo] == y) r = y >= x ? lo - diag[x] : ntpos[rb + lo] - diag[y];
            if (r < 0) atomicOr(ovf, 1);
            if (r > 65535) atomicOr(ovf, 2);
            klr[(int64_t)(a * 3 + b) * n + i] = (uint16_t)min(max(r, 0), 65535);
        }
    }
}

__global__ void k_list_kl(const int* __restrict__ ids, int64_t n, const int* __restrict__ pk,
                          const int* __restrict__ pl, int2* __restrict__ kl) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = ids[i];
    kl[i] = make_int2(pk[p], pl[p]);
}

__global__ void k_max_deg(const int* ne_ptr, int64_t M, int* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    warp_atomic_max(out, i < M ? ne_ptr[i + 1] - ne_ptr[i] : 0);
}

void build_bulk_index(Mesh& m, PairCache& pc, cudaStream_t st) {
    const int64_t K = m.K;
    DBuf<int> ovf;
    ovf.alloc(1, st);
    ovf.zero(st);
    pc.epos.alloc(K * 8, st);
    k_epos<<<nblk(K, 256), 256, 0, st>>>(m.T.p, K, pc.nrow_ptr.p, pc.ncol.p, pc.up_start.p, pc.epos.p, ovf.p);
    NLFEM_LAUNCH_CHECK();
    pc.klr_whole.alloc(pc.nwhole * 9, st);
    pc.klr_cut.alloc(pc.ncut * 9, st);
    // the elements of every whole-pair list entry: the whole-pair kernel's first loads then do
    // not wait on the pair ids (the cut-pair kernel, bound elsewhere, gained nothing from it)
    pc.kl_whole.alloc(pc.nwhole, st);
    if (pc.nwhole > 0) {
        k_list_kl<<<nblk(pc.nwhole, 256), 256, 0, st>>>(pc.whole_ids.p, pc.nwhole, pc.pk.p, pc.pl.p, pc.kl_whole.p);
        NLFEM_LAUNCH_CHECK();
    }
    DBuf<int> diag;
    diag.alloc(m.M, st);
    k_diag<<<nblk(m.M, 256), 256, 0, st>>>(pc.nrow_ptr.p, pc.ncol.p, m.M, diag.p);
    NLFEM_LAUNCH_CHECK();
    if (pc.nwhole > 0) {
        k_klr<<<nblk(pc.nwhole, 256), 256, 0, st>>>(pc.whole_ids.p, pc.nwhole, pc.pk.p, pc.pl.p, m.T.p, pc.nrow_ptr.p,
                                                    pc.ncol.p, pc.ntpos.p, diag.p, pc.klr_whole.p, ovf.p);
        NLFEM_LAUNCH_CHECK();
    }
    if (pc.ncut > 0) {
        k_klr<<<nblk(pc.ncut, 256), 256, 0, st>>>(pc.cut_ids.p, pc.ncut, pc.pk.p, pc.pl.p, m.T.p, pc.nrow_ptr.p,
                                                  pc.ncol.p, pc.ntpos.p, diag.p, pc.klr_cut.p, ovf.p);
        NLFEM_LAUNCH_CHECK();
    }
    // bound on the values added into one entry: every pair with the node in E_k or in E_l
    // adds at most three values (kk, ll, kl) into a diagonal entry, fewer elsewhere
    DBuf<int> md;
    md.alloc(1, st);
    md.zero(st);
    k_max_deg<<<nblk(m.M, 256), 256, 0, st>>>(m.ne_ptr.p, m.M, md.p);
    NLFEM_LAUNCH_CHECK();
    int h[2] = {0, 0};
    NLFEM_CUDA_TRY(cudaMemcpyAsync(&h[0], ovf.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    NLFEM_CUDA_TRY(cudaMemcpyAsync(&h[1], md.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
    NLFEM_CHECK(!(h[0] & 1), NLFEM_ERR_CUDA, "internal error: a pair's node pair is missing from the CSR pattern");
    NLFEM_CHECK(!(h[0] & 2), NLFEM_ERR_UNSUPPORTED, "a CSR row has more than 65536 upper entries");
    NLFEM_CHECK(!(h[0] & 4), NLFEM_ERR_UNSUPPORTED, "more than 2^31 upper CSR entries");
    const int64_t maxp = std::max(max_segment_i64(pc.pair_ptr.p, K, st), max_segment_i64(pc.pT_ptr.p, K, st));
    pc.acc_terms = 3 * (int64_t)std::max(h[1], 1) * 2 * std::max<int64_t>(maxp, 1);
    pc.ntpos.release();
}

// fixed-point upper entries -> CSR values (and their mirrors); warp per node row
template <int NDOF>
__global__ void k_acc_to_csr(int64_t M, const int64_t* __restrict__ nptr, const int* __restrict__ ncol,
                             const int64_t* __restrict__ up_start, const unsigned long long* __restrict__ acc,
                             const FixState* __restrict__ fix, const int64_t* __restrict__ row_ptr,
                             const int64_t* __restrict__ tpos, double* __restrict__ val) {
    constexpr int NC = NDOF == 1 ? 1 : 3;
    const double inv_scale = ldexp(1.0, -fix->shift);
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= M) return;
    const int64_t b = nptr[i], e = nptr[i + 1];
    // position of the diagonal: the first column >= i
    int64_t a = b, c = e;
    while (a < c) {
        const int64_t mid = (a + c) >> 1;
        if (ncol[mid] < (int)i) a = mid + 1;
        else c = mid;
    }
    const int64_t td = a, u0 = up_start[i];
    for (int64_t t = td + lane; t < e; t += 32) {
        const int64_t u = u0 + (t - td);
        double v[NC];
#pragma unroll
        for (int q = 0; q < NC; ++q) v[q] = (double)(long long)acc[u * NC + q] * inv_scale;
        if (NDOF == 1) {
            const int64_t s = row_ptr[i] + (t - b);
            val[s] = v[0];
            val[tpos[s]] = v[0];
        } else {
            const int j = ncol[t];
            const int64_t r = t - b;
            const double comp[4] = {v[0], v[1], v[1], v[2]};  // xx, xy, yx, yy
            for (int c1 = 0; c1 < 2; ++c1)
                for (int c2 = 0; c2 < 2; ++c2) {
                    if (j == (int)i && c2 < c1) continue;  // the diagonal node block: upper dofs only
                    const int64_t s = row_ptr[i * 2 + c1] + 2 * r + c2;
                    val[s] = comp[c1 * 2 + c2];
                    val[tpos[s]] = comp[c1 * 2 + c2];
                }
        }
    }
}

void run_reduction(Mesh& m, PairCache& pc, const Params& prm, System& sys, cudaStream_t st) {
    if (prm.precision == NLFEM_PREC_FP32_BULK) {
        // every upper entry is written with its mirror, so val needs no clearing
        const unsigned g = nblk(m.M * 32, 256);
        if (m.M == 0) return;
        if (pc.ndof == 1)
            k_acc_to_csr<1><<<g, 256, 0, st>>>(m.M, pc.nrow_ptr.p, pc.ncol.p, pc.up_start.p, sys.acc.p, sys.fix.p,
                                               pc.row_ptr.p, pc.tpos.p, sys.val.p);
        else
            k_acc_to_csr<2><<<g, 256, 0, st>>>(m.M, pc.nrow_ptr.p, pc.ncol.p, pc.up_start.p, sys.acc.p, sys.fix.p,
                                               pc.row_ptr.p, pc.tpos.p, sys.val.p);
        NLFEM_LAUNCH_CHECK();
        return;
    }
    if (!pc.slots_built) build_slots(m, pc, st);
    NLFEM_CUDA_TRY(cudaMemsetAsync(sys.val.p, 0, sys.val.bytes(), st));
    if (pc.n_upper == 0) return;
    // half a warp per entry, blocks dispatched in order: the entries in flight stay a compact
    // band of the strip-ordered rows (a grid-stride loop would scatter them over the mesh)
    const unsigned g = (unsigned)std::min<int64_t>(nblk(pc.n_upper * 16, 256), 0x7fffffffll);
    if (pc.ndof == 1)
        k_reduce<double, 1><<<g, 256, 0, st>>>(pc.n_upper, pc.up_pos.p, pc.up_row.p, pc.nrow_ptr.p, pc.ncol.p,
                                               pc.seg_ptr.p, pc.idx.p, pc.pbase.p, sys.contrib64.p, pc.row_ptr.p,
                                               pc.tpos.p, sys.val.p);
    else
        k_reduce<double, 2><<<g, 256, 0, st>>>(pc.n_upper, pc.up_pos.p, pc.up_row.p, pc.nrow_ptr.p, pc.ncol.p,
                                               pc.seg_ptr.p, pc.idx.p, pc.pbase.p, sys.contrib64.p, pc.row_ptr.p,
                                               pc.tpos.p, sys.val.p);
    NLFEM_LAUNCH_CHECK();
}

}  // namespace nlfem
