// Solve of the nonlocal Dirichlet problem (eq. inhomogeneousDirichletData):
//   A_FF u_F = F_F - A_FD g,
// with the columns of A split into free dofs and Dirichlet dofs. The paper returns the
// CSR matrix and leaves the solve to the user; here conjugate gradients run in FP32
// on A_FF inside an FP64 residual-refinement loop, which recovers FP64 accuracy of u_F.
// All scalars (alpha, beta, residual norms) stay on the device; the host reads the
// residual only every CHECK_EVERY iterations. Dot products are reduced in a fixed order.
// A block of CHECK_EVERY inner iterations is a fixed sequence of launches on fixed buffers:
// it is captured once per system into a CUDA graph and replayed, which removes the
// per-launch host cost that dominates small solves; the kernels and their order are the
// same, so the results are the same bits.
#include <algorithm>
#include <cmath>

#include "nlfem_internal.cuh"

namespace nlfem {

static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

struct SolveState {
    int64_t N = 0;
    DBuf<float> val32;    // FP32 copy of A
    DBuf<int8_t> freem;   // dof is free
    DBuf<double> b, x, r64, y64;
    DBuf<float> r, p, q, d;
    DBuf<double> part;    // partial sums of dot products
    DBuf<unsigned> ticket;  // blocks done of the running fused CG kernel (0 between launches)
    DBuf<double> sc;      // device scalars: [0] rho, [1] p.q, [2] rho_new, [3] |r64|^2, [4] |b|^2,
                          // [5] beta (Dirichlet iteration), [8..10] null-space coefficients,
                          // [11] Gram-Schmidt scratch
    DBuf<double> Z;       // orthonormal null-space basis of the full matrix [nz][N] (Neumann solve)
    int nz = 0;
    cudaStream_t cap = nullptr;                   // private stream the blocks are captured on
    cudaGraphExec_t blk[2] = {nullptr, nullptr};  // [0] Dirichlet block, [1] Neumann block
    ~SolveState() {
        for (auto& g : blk)
            if (g) cudaGraphExecDestroy(g);
        if (cap) cudaStreamDestroy(cap);
    }
};

// Runs body(stream) on st: the first time it is captured from a private stream into W.blk[kind],
// every time the graph is launched on st. body must enqueue only kernels on the stream it is
// given, on buffers that stay in place for the life of W.
template <typename F>
static void run_block(SolveState& W, int kind, F&& body, cudaStream_t st) {
    if (!W.blk[kind]) {
        if (!W.cap) NLFEM_CUDA_TRY(cudaStreamCreateWithFlags(&W.cap, cudaStreamNonBlocking));
        NLFEM_CUDA_TRY(cudaStreamBeginCapture(W.cap, cudaStreamCaptureModeThreadLocal));
        cudaGraph_t g = nullptr;
        try {
            body(W.cap);
        } catch (...) {
            cudaStreamEndCapture(W.cap, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        NLFEM_CUDA_TRY(cudaStreamEndCapture(W.cap, &g));
        cudaGraphExec_t ex = nullptr;
        const cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        NLFEM_CUDA_TRY(e);
        W.blk[kind] = ex;
    }
    NLFEM_CUDA_TRY(cudaGraphLaunch(W.blk[kind], st));
}

static constexpr int DOT_BLOCKS = 1024;
static constexpr int DOT_THREADS = 256;

__global__ void k_to_f32(const double* a, float* b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

__global__ void k_freemask(const int8_t* dir, int64_t N, int ndof, int8_t* freem) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) freem[i] = dir[i / ndof] ? 0 : 1;
}

// y = A x on free rows (x is zero at Dirichlet dofs); warp per row, fixed shuffle tree
template <typename T, typename V>
__global__ void k_spmv(const int64_t* rp, const int* col, const V* val, const T* x, T* y, const int8_t* freem,
                       int64_t N) {
    int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (i >= N) return;
    const bool fr = !freem || freem[i];   // freem == nullptr: every dof is unknown (Neumann solve)
    T s = 0;
    if (fr)
        for (int64_t t = rp[i] + lane; t < rp[i + 1]; t += 32) s += (T)val[t] * x[col[t]];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[i] = fr ? s : (T)0;
}

// b = F - A x with x = g at Dirichlet dofs and 0 elsewhere; zero at Dirichlet rows
__global__ void k_rhs(const int64_t* rp, const int* col, const double* val, const double* g, const double* F,
                      const int8_t* freem, double* b, int64_t N) {
    int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (i >= N) return;
    double s = 0;
    if (freem[i] && g)
        for (int64_t t = rp[i] + lane; t < rp[i + 1]; t += 32) {
            int j = col[t];
            if (!freem[j]) s += val[t] * g[j];
        }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) b[i] = freem[i] ? F[i] - s : 0.0;
}

template <typename T1, typename T2>
__global__ void k_dot_part(const T1* a, const T2* b, int64_t n, double* part) {
    __shared__ double sh[DOT_THREADS];
    double s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += (double)a[i] * (double)b[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = DOT_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_dot_final(const double* part, double* out) {
    __shared__ double sh[DOT_BLOCKS];
    for (int i = threadIdx.x; i < DOT_BLOCKS; i += blockDim.x) sh[i] = part[i];
    __syncthreads();
    for (int o = DOT_BLOCKS / 2; o > 0; o >>= 1) {
        for (int i = threadIdx.x; i < o; i += blockDim.x) sh[i] += sh[i + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

template <typename T1, typename T2>
static void dot(const T1* a, const T2* b, int64_t n, double* part, double* out, cudaStream_t st) {
    k_dot_part<T1, T2><<<DOT_BLOCKS, DOT_THREADS, 0, st>>>(a, b, n, part);
    k_dot_final<<<1, 1024, 0, st>>>(part, out);
}

// CG updates with device scalars: alpha = rho / pq
__global__ void k_cg_update(float* d, float* r, const float* p, const float* q, const double* sc, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double pq = sc[1];
    float alpha = pq != 0.0 ? (float)(sc[0] / pq) : 0.f;
    d[i] += alpha * p[i];
    r[i] -= alpha * q[i];
}

__global__ void k_cg_dir(float* p, const float* r, double* sc, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float beta = sc[0] != 0.0 ? (float)(sc[2] / sc[0]) : 0.f;
    p[i] = r[i] + beta * p[i];
}

__global__ void k_roll(double* sc) { sc[0] = sc[2]; }

// ---- one CG iteration in three kernels (Dirichlet solve) ----------------------------------
// Each kernel reduces its dot product in the same launch: every block writes its partial sum,
// and the last block to finish (a ticket counter) adds the partials in block order, so the
// sum is the same on every run. The grids depend on N only (the product: one warp per row).
static constexpr int CG_THREADS = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = CG_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// partial sum of this block into part[blockIdx.x]; true in every thread of the last block,
// which then holds in sh the total of all partials (block order, then a fixed tree)
__device__ __forceinline__ bool reduce_last(double v, double* part, unsigned* ticket, double* sh, double& total) {
    __shared__ bool last;
    const double b = block_sum(v, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = b;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    double t = 0;
    for (unsigned j = threadIdx.x; j < gridDim.x; j += CG_THREADS) t += __ldcg(part + j);
    total = block_sum(t, sh);
    if (threadIdx.x == 0) *ticket = 0;
    return true;
}

// q = A_FF p (warp per row), sc[1] = p . q
__global__ void __launch_bounds__(CG_THREADS) k_cg_spmv_pq(const int64_t* __restrict__ rp, const int* __restrict__ col,
                                                           const float* __restrict__ val, const float* __restrict__ p,
                                                           float* __restrict__ q, const int8_t* __restrict__ freem,
                                                           int64_t N, double* part, unsigned* ticket, double* sc) {
    __shared__ double sh[CG_THREADS];
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (CG_THREADS / 32);
    double acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * (CG_THREADS / 32) + (threadIdx.x >> 5); i < N; i += nw) {
        const bool fr = freem[i];
        float s = 0;
        if (fr)
            for (int64_t t = rp[i] + lane; t < rp[i + 1]; t += 32) s += val[t] * p[col[t]];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const float qi = fr ? s : 0.f;
            q[i] = qi;
            acc += (double)p[i] * (double)qi;
        }
    }
    double total;
    if (reduce_last(acc, part, ticket, sh, total) && threadIdx.x == 0) sc[1] = total;
}

// alpha = sc[0] / sc[1]; d += alpha p; r -= alpha q; rho_new = r . r;
// then sc[5] = beta = rho_new / sc[0] and sc[0] = rho_new
__global__ void __launch_bounds__(CG_THREADS) k_cg_update_rr(float* __restrict__ d, float* __restrict__ r,
                                                             const float* __restrict__ p, const float* __restrict__ q,
                                                             int64_t N, double* part, unsigned* ticket, double* sc) {
    __shared__ double sh[CG_THREADS];
    const double rho = sc[0], pq = sc[1];
    const float alpha = pq != 0.0 ? (float)(rho / pq) : 0.f;
    double acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * CG_THREADS + threadIdx.x; i < N; i += (int64_t)gridDim.x * CG_THREADS) {
        d[i] += alpha * p[i];
        const float ri = r[i] - alpha * q[i];
        r[i] = ri;
        acc += (double)ri * (double)ri;
    }
    double total;
    if (reduce_last(acc, part, ticket, sh, total) && threadIdx.x == 0) {
        sc[2] = total;
        sc[5] = rho != 0.0 ? total / rho : 0.0;
        sc[0] = total;
    }
}

// p = r + beta p
__global__ void k_cg_dir_b(float* __restrict__ p, const float* __restrict__ r, const double* __restrict__ sc, int64_t N) {
    const float beta = (float)sc[5];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = r[i] + beta * p[i];
}

__global__ void k_start(float* r, float* p, float* d, const double* r64, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v = (float)r64[i];
    r[i] = v;
    p[i] = v;
    d[i] = 0.f;
}

__global__ void k_add_corr(double* x, const float* d, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += (double)d[i];
}

__global__ void k_sub(const double* b, const double* y, double* r, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = b[i] - y[i];
}

__global__ void k_final_u(const double* x, const double* g, const int8_t* freem, double* u, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) u[i] = freem[i] ? x[i] : (g ? g[i] : 0.0);
}

// ---- pure Neumann-type solve on the full matrix ------------------------------------------
// The full matrix annihilates the constants (scalar kernels) and the rigid motions (vector
// peridynamic kernel) up to rounding: the symmetrised form of Rem. 2.4. The solve returns the
// u orthogonal to that null space N with P A u = P F, P the orthogonal projector onto the
// complement of N, by conjugate gradients on P A P (every residual projected) inside the same
// FP64 refinement as the Dirichlet solve.

// raw basis: ones, or for two dofs per node the translations and the rotation (-(y - cy), x - cx)
__global__ void k_null_raw(const double2* X, int64_t M, int ndof, double cx, double cy, double* Z, int64_t N) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    if (ndof == 1) {
        Z[i] = 1.0;
        return;
    }
    const double x = X[i].x - cx, y = X[i].y - cy;
    Z[2 * i] = 1.0;
    Z[2 * i + 1] = 0.0;
    Z[N + 2 * i] = 0.0;
    Z[N + 2 * i + 1] = 1.0;
    Z[2 * N + 2 * i] = -y;
    Z[2 * N + 2 * i + 1] = x;
}

// a -= c b with c read from the device (Gram-Schmidt step)
__global__ void k_axpy_dev(double* a, const double* b, const double* c, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] -= *c * b[i];
}

__global__ void k_normalise(double* a, const double* nn, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] /= sqrt(*nn);
}

// v -= sum_j c_j Z_j, the coefficients c_j = Z_j . v read from the device
template <typename T>
__global__ void k_project_out(T* v, const double* Z, const double* c, int nz, int64_t N) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double s = (double)v[i];
    for (int j = 0; j < nz; ++j) s -= c[j] * Z[(int64_t)j * N + i];
    v[i] = (T)s;
}

template <typename T>
static void project_out(SolveState& W, T* v, cudaStream_t st) {
    for (int j = 0; j < W.nz; ++j) dot(W.Z.p + (int64_t)j * W.N, v, W.N, W.part.p, W.sc.p + 8 + j, st);
    k_project_out<T><<<nblk(W.N, 256), 256, 0, st>>>(v, W.Z.p, W.sc.p + 8, W.nz, W.N);
}

static int ensure_solver(System& S, cudaStream_t st) {
    if (S.solver) return NLFEM_OK;
    const int64_t N = S.N;
    auto ss = std::make_shared<SolveState>();
    ss->N = N;
    ss->val32.alloc(S.nnz, st);
    k_to_f32<<<nblk(S.nnz, 256), 256, 0, st>>>(S.val.p, ss->val32.p, S.nnz);
    NLFEM_LAUNCH_CHECK();
    ss->freem.alloc(N, st);
    k_freemask<<<nblk(N, 256), 256, 0, st>>>(S.mesh->dir.p, N, S.prm.ndof, ss->freem.p);
    NLFEM_LAUNCH_CHECK();
    ss->b.alloc(N, st); ss->x.alloc(N, st); ss->r64.alloc(N, st); ss->y64.alloc(N, st);
    ss->r.alloc(N, st); ss->p.alloc(N, st); ss->q.alloc(N, st); ss->d.alloc(N, st);
    // partial sums: DOT_BLOCKS for dot(), a block's share of the fused CG kernels (warp per row)
    ss->part.alloc(std::max<int64_t>(DOT_BLOCKS, nblk(N * 32, CG_THREADS)), st);
    ss->ticket.alloc(1, st);
    ss->ticket.zero(st);
    ss->sc.alloc(16, st);
    S.solver = ss;
    return NLFEM_OK;
}

int solve_neumann(System& S, double tol, int max_iter, double* u_out, nlfem_solve_info* info, cudaStream_t st) {
    int rc = ensure_solver(S, st);
    if (rc) return rc;
    const int64_t N = S.N;
    PairCache& pc = *S.pc;
    SolveState& W = *S.solver;
    const unsigned gw = nblk(N * 32, 256), ge = nblk(N, 256);
    if (!W.nz) {
        const Mesh& m = *S.mesh;
        W.nz = S.prm.ndof == 1 ? 1 : 3;
        W.Z.alloc((size_t)W.nz * N, st);
        k_null_raw<<<nblk(m.M, 256), 256, 0, st>>>(m.X.p, m.M, S.prm.ndof, 0.5 * (m.bbox[0] + m.bbox[2]),
                                                 0.5 * (m.bbox[1] + m.bbox[3]), W.Z.p, N);
        NLFEM_LAUNCH_CHECK();
        // modified Gram-Schmidt in FP64
        for (int k = 0; k < W.nz; ++k) {
            double* zk = W.Z.p + (int64_t)k * N;
            for (int j = 0; j < k; ++j) {
                const double* zj = W.Z.p + (int64_t)j * N;
                dot(zj, zk, N, W.part.p, W.sc.p + 11, st);
                k_axpy_dev<<<ge, 256, 0, st>>>(zk, zj, W.sc.p + 11, N);
            }
            dot(zk, zk, N, W.part.p, W.sc.p + 11, st);
            k_normalise<<<ge, 256, 0, st>>>(zk, W.sc.p + 11, N);
            NLFEM_LAUNCH_CHECK();
        }
    }
    // b = P F
    NLFEM_CUDA_TRY(cudaMemcpyAsync(W.b.p, S.F.p, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    project_out(W, W.b.p, st);
    W.x.zero(st);
    dot(W.b.p, W.b.p, N, W.part.p, W.sc.p + 4, st);
    NLFEM_CUDA_TRY(cudaMemcpyAsync(W.r64.p, W.b.p, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    NLFEM_LAUNCH_CHECK();
    double bb = 0;
    NLFEM_CUDA_TRY(cudaMemcpyAsync(&bb, W.sc.p + 4, sizeof bb, cudaMemcpyDeviceToHost, st));
    NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
    const double bnorm = std::sqrt(bb);
    int iters = 0, refs = 0;
    double rel = bnorm > 0 ? 1.0 : 0.0;
    const int CHECK_EVERY = 8;
    while (rel > tol && iters < max_iter) {
        k_start<<<ge, 256, 0, st>>>(W.r.p, W.p.p, W.d.p, W.r64.p, N);
        NLFEM_LAUNCH_CHECK();
        dot(W.r.p, W.r.p, N, W.part.p, W.sc.p + 0, st);
        double rho0 = 0;
        NLFEM_CUDA_TRY(cudaMemcpyAsync(&rho0, W.sc.p, sizeof rho0, cudaMemcpyDeviceToHost, st));
        NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
        const double inner_tol2 = rho0 * 1e-8;
        auto iterate = [&](cudaStream_t s, int n) {
            for (int j = 0; j < n; ++j) {
                k_spmv<float, float><<<gw, 256, 0, s>>>(pc.row_ptr.p, pc.col.p, W.val32.p, W.p.p, W.q.p, nullptr, N);
                dot(W.p.p, W.q.p, N, W.part.p, W.sc.p + 1, s);
                k_cg_update<<<ge, 256, 0, s>>>(W.d.p, W.r.p, W.p.p, W.q.p, W.sc.p, N);
                project_out(W, W.r.p, s);
                dot(W.r.p, W.r.p, N, W.part.p, W.sc.p + 2, s);
                k_cg_dir<<<ge, 256, 0, s>>>(W.p.p, W.r.p, W.sc.p, N);
                k_roll<<<1, 1, 0, s>>>(W.sc.p);
                NLFEM_LAUNCH_CHECK();
            }
        };
        int it = 0;
        while (iters < max_iter) {
            const int n = std::min(CHECK_EVERY, max_iter - iters);
            if (n == CHECK_EVERY)
                run_block(W, 1, [&](cudaStream_t s) { iterate(s, CHECK_EVERY); }, st);
            else
                iterate(st, n);
            it += n;
            iters += n;
            if (n == CHECK_EVERY) {
                double rho = 0;
                NLFEM_CUDA_TRY(cudaMemcpyAsync(&rho, W.sc.p, sizeof rho, cudaMemcpyDeviceToHost, st));
                NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
                if (!(rho > inner_tol2) || it >= 2000) break;
            }
        }
        // x += d, kept orthogonal to N; r64 = P (b - A x) in FP64
        k_add_corr<<<ge, 256, 0, st>>>(W.x.p, W.d.p, N);
        project_out(W, W.x.p, st);
        k_spmv<double, double><<<gw, 256, 0, st>>>(pc.row_ptr.p, pc.col.p, S.val.p, W.x.p, W.y64.p, nullptr, N);
        k_sub<<<ge, 256, 0, st>>>(W.b.p, W.y64.p, W.r64.p, N);
        project_out(W, W.r64.p, st);
        NLFEM_LAUNCH_CHECK();
        dot(W.r64.p, W.r64.p, N, W.part.p, W.sc.p + 3, st);
        double rr = 0;
        NLFEM_CUDA_TRY(cudaMemcpyAsync(&rr, W.sc.p + 3, sizeof rr, cudaMemcpyDeviceToHost, st));
        NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
        rel = bnorm > 0 ? std::sqrt(rr) / bnorm : 0.0;
        ++refs;
        if (refs > 50) break;
    }
    NLFEM_CUDA_TRY(cudaMemcpyAsync(u_out, W.x.p, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
    if (info) {
        info->iterations = iters;
        info->refinements = refs;
        info->rel_residual = rel;
    }
    if (rel > tol) {
        set_error("projected CG did not reach the tolerance: relative residual " + std::to_string(rel));
        return NLFEM_ERR_NOT_CONVERGED;
    }
    return NLFEM_OK;
}

int solve_system(System& S, const double* g, double tol, int max_iter, double* u_out, nlfem_solve_info* info,
                 cudaStream_t st) {
    int rc = ensure_solver(S, st);
    if (rc) return rc;
    const int64_t N = S.N;
    PairCache& pc = *S.pc;
    SolveState& W = *S.solver;
    const unsigned gw = nblk(N * 32, 256), ge = nblk(N, 256);
    k_rhs<<<gw, 256, 0, st>>>(pc.row_ptr.p, pc.col.p, S.val.p, g, S.F.p, W.freem.p, W.b.p, N);
    NLFEM_LAUNCH_CHECK();
    W.x.zero(st);
    dot(W.b.p, W.b.p, N, W.part.p, W.sc.p + 4, st);
    NLFEM_CUDA_TRY(cudaMemcpyAsync(W.r64.p, W.b.p, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    double bb = 0;
    NLFEM_CUDA_TRY(cudaMemcpyAsync(&bb, W.sc.p + 4, sizeof bb, cudaMemcpyDeviceToHost, st));
    NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
    const double bnorm = std::sqrt(bb);
    int iters = 0, refs = 0;
    double rel = bnorm > 0 ? 1.0 : 0.0;
    const int CHECK_EVERY = 8;
    while (rel > tol && iters < max_iter) {
        // inner FP32 CG on A_FF d = r64, to a relative tolerance of 1e-4 of |r64|
        k_start<<<ge, 256, 0, st>>>(W.r.p, W.p.p, W.d.p, W.r64.p, N);
        NLFEM_LAUNCH_CHECK();
        dot(W.r.p, W.r.p, N, W.part.p, W.sc.p + 0, st);
        double rho0 = 0;
        NLFEM_CUDA_TRY(cudaMemcpyAsync(&rho0, W.sc.p, sizeof rho0, cudaMemcpyDeviceToHost, st));
        NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
        const double inner_tol2 = rho0 * 1e-8;
        const unsigned gq = gw, gu = std::min<unsigned>(ge, DOT_BLOCKS);  // one row per warp for the product
        auto iterate = [&](cudaStream_t s, int n) {
            for (int j = 0; j < n; ++j) {
                k_cg_spmv_pq<<<gq, CG_THREADS, 0, s>>>(pc.row_ptr.p, pc.col.p, W.val32.p, W.p.p, W.q.p, W.freem.p, N,
                                                       W.part.p, W.ticket.p, W.sc.p);
                k_cg_update_rr<<<gu, CG_THREADS, 0, s>>>(W.d.p, W.r.p, W.p.p, W.q.p, N, W.part.p, W.ticket.p, W.sc.p);
                k_cg_dir_b<<<gu, 256, 0, s>>>(W.p.p, W.r.p, W.sc.p, N);
                NLFEM_LAUNCH_CHECK();
            }
        };
        int it = 0;
        while (iters < max_iter) {
            const int n = std::min(CHECK_EVERY, max_iter - iters);
            if (n == CHECK_EVERY)
                run_block(W, 0, [&](cudaStream_t s) { iterate(s, CHECK_EVERY); }, st);
            else
                iterate(st, n);
            it += n;
            iters += n;
            if (n == CHECK_EVERY) {
                double rho = 0;
                NLFEM_CUDA_TRY(cudaMemcpyAsync(&rho, W.sc.p, sizeof rho, cudaMemcpyDeviceToHost, st));
                NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
                if (!(rho > inner_tol2) || it >= 2000) break;
            }
        }
        // x += d; r64 = b - A_FF x in FP64
        k_add_corr<<<ge, 256, 0, st>>>(W.x.p, W.d.p, N);
        k_spmv<double, double><<<gw, 256, 0, st>>>(pc.row_ptr.p, pc.col.p, S.val.p, W.x.p, W.y64.p, W.freem.p, N);
        k_sub<<<ge, 256, 0, st>>>(W.b.p, W.y64.p, W.r64.p, N);
        NLFEM_LAUNCH_CHECK();
        dot(W.r64.p, W.r64.p, N, W.part.p, W.sc.p + 3, st);
        double rr = 0;
        NLFEM_CUDA_TRY(cudaMemcpyAsync(&rr, W.sc.p + 3, sizeof rr, cudaMemcpyDeviceToHost, st));
        NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
        rel = std::sqrt(rr) / bnorm;
        ++refs;
        if (refs > 50) break;
    }
    k_final_u<<<ge, 256, 0, st>>>(W.x.p, g, W.freem.p, u_out, N);
    NLFEM_LAUNCH_CHECK();
    NLFEM_CUDA_TRY(cudaStreamSynchronize(st));
    if (info) {
        info->iterations = iters;
        info->refinements = refs;
        info->rel_residual = rel;
    }
    if (rel > tol) {
        set_error("CG did not reach the tolerance: relative residual " + std::to_string(rel));
        return NLFEM_ERR_NOT_CONVERGED;
    }
    return NLFEM_OK;
}

}  // namespace nlfem
