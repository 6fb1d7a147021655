// Tail of the V-cycle in one launch.
//
// The coarse levels of the hierarchy are too small to fill the GPU: a colour
// pass on a 16^3 level costs the same few microseconds of launch and memory
// latency as one on a 64^3 level.  From the first level with at most
// kTailCells cells down to the dense coarsest solve and back up, this kernel
// runs every step of the V-cycle (Sec. 3.7.3: pre-smoothing, restriction of
// the residual, the coarsest solve, prolongation, post-smoothing) in one
// block of 1024 threads, with a block barrier between steps.  Each cell
// update, restriction sum, prolongation and the dense solve use the same
// arithmetic in the same order as the separate kernels, so the result is the
// same bit for bit.
#include "kernels.cuh"

namespace paris {

namespace {

constexpr int kTailThreads = 1024;

// One element from global to shared memory without a register round trip
// (cp.async; completed by cp.async.wait_all).  Both addresses are aligned to
// the element size.
__device__ __forceinline__ void async_copy(float* dst, const float* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void async_copy(double* dst, const double* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}

template <typename T>
struct TailArgs {
    int n;                    // levels in the tail, the last one the dense coarsest
    TailLevel<T> L[kMaxTail];
    const double* Minv;       // dense inverse of the coarsest operator
    T omega;
    int nu1, nu2;
};

// t / n by the multiplier m of TailLevel (exact for t, n < 2^16)
__device__ __forceinline__ unsigned udiv(unsigned t, unsigned n, unsigned m) { return n == 1 ? t : __umulhi(t, m); }

// (i, j, k) of index t on an n0 x n1 x n2 box, x fastest (m0, m1: the multipliers of n0, n1)
__device__ __forceinline__ void tail_split(unsigned t, unsigned n0, unsigned n1, unsigned m0, unsigned m1, int& i,
                                           int& j, int& k) {
    const unsigned row = udiv(t, n0, m0);
    i = (int)(t - row * n0);
    const unsigned kk = udiv(row, n1, m1);
    j = (int)(row - kk * n1);
    k = (int)kk;
}

// One colour pass of over-relaxed red-black Gauss-Seidel on a tail level (the
// update of rbgs_kernel; zero: x taken as 0, the other colour zeroed).
template <typename T, bool USEW>
__device__ void tail_pass(const TailLevel<T> L, int color, bool zero, T omega) {
    const Geo g = L.g;
    const T hs = T(1) / L.scale;
    const int npair = (g.nx + 1) / 2;
    const int total = npair * g.ny * g.nz;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        int tp, j, k;
        tail_split((unsigned)t, (unsigned)npair, (unsigned)g.ny, L.mp, L.my, tp, j, k);
        const int i0 = 2 * tp;
        const int i = i0 + ((i0 + j + k + color) & 1);
        const int io = i0 + 1 - (i - i0);
        if (i < g.nx) {
            Stencil<T> s;
            int c;
            load_stencil_fast<T>(g, L.bx, L.by, L.bz, i, j, k, s, c);
            T xn;
            if (zero) {
                const T wc = USEW ? L.w[c] : inv_sum6(s.b);
                xn = omega * wc * (L.f[c] * hs);
            } else {
                T acc = L.f[c] * hs;
#pragma unroll
                for (int q = 0; q < 6; ++q) acc = fma(s.b[q], L.x[s.nb[q]], acc);
                const T xc = L.x[c];
                xn = fma(omega, fma(USEW ? L.w[c] : inv_sum6(s.b), acc, -xc), xc);
            }
            L.x[c] = xn;
        }
        if (zero && io < g.nx) L.x[g.cidx(io, j, k)] = T(0);
    }
}

template <typename T, bool USEW>
__device__ void tail_smooth(const TailLevel<T> L, int sweeps, bool first_zero, bool reverse, T omega) {
    const int c0 = reverse ? 1 : 0;
    for (int s = 0; s < sweeps; ++s) {
        tail_pass<T, USEW>(L, c0, first_zero && s == 0, omega);
        __syncthreads();
        tail_pass<T, USEW>(L, 1 - c0, false, omega);
        __syncthreads();
    }
}

// coarse f = average over the children of the fine residual f - A x (A x on
// the coarse cell's surface faces, as restrict_residual_kernel)
template <typename T>
__device__ void tail_restrict(const TailLevel<T> F, const TailLevel<T> C) {
    const Geo fg = F.g;
    const Geo cg = C.g;
    const int fa0 = C.fac[0], fa1 = C.fac[1], fa2 = C.fac[2];
    const int total = cg.nx * cg.ny * cg.nz;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        int I, J, K;
        tail_split((unsigned)t, (unsigned)cg.nx, (unsigned)cg.ny, C.mx, C.my, I, J, K);
        T sum = T(0);
        for (int dk = 0; dk < fa2; ++dk)
            for (int dj = 0; dj < fa1; ++dj)
                for (int di = 0; di < fa0; ++di) {
                    const int i = I * fa0 + di, j = J * fa1 + dj, k = K * fa2 + dk;
                    Stencil<T> s;
                    int c;
                    load_stencil_fast<T>(fg, F.bx, F.by, F.bz, i, j, k, s, c);
                    sum += F.f[c] - apply_A_faces(s, F.x, F.x[c], F.scale, surface_faces(di, dj, dk, fa0, fa1, fa2));
                }
        C.f[t] = sum / T(fa0 * fa1 * fa2);
    }
}

// x_fine += x_coarse[parent]
template <typename T>
__device__ void tail_prolong(const TailLevel<T> C, const TailLevel<T> F) {
    const Geo fg = F.g;
    const Geo cg = C.g;
    const int total = fg.nx * fg.ny * fg.nz;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        int i, j, k;
        tail_split((unsigned)t, (unsigned)fg.nx, (unsigned)fg.ny, F.mx, F.my, i, j, k);
        F.x[t] += C.x[cg.cidx(i >> (C.fac[0] - 1), j >> (C.fac[1] - 1), k >> (C.fac[2] - 1))];
    }
}

// x = M (f - mean f) on the coarsest level (FP64 arithmetic)
template <typename T>
__device__ void tail_coarse_solve(const TailLevel<T> L, const double* __restrict__ M, double* fs,
                                  double* mean) {
    const int n = L.g.nx * L.g.ny * L.g.nz;
    for (int c = threadIdx.x; c < n; c += blockDim.x) fs[c] = (double)L.f[c];
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int c = 0; c < n; ++c) t += fs[c];
        *mean = t / (double)n;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < n; ++c) acc = fma(M[r * n + c], fs[c] - *mean, acc);
        L.x[r] = (T)acc;
    }
}

// SMEM: the levels' coefficients, inverse diagonals, right-hand sides and
// solutions and the dense inverse are staged in shared memory; only the first
// level's solution is written back (its right-hand side came from above).
// The level table itself lives in shared memory (Ls), pointing at either copy.
template <typename T, bool USEW, bool SMEM>
__global__ void __launch_bounds__(kTailThreads) tail_vcycle_kernel(const __grid_constant__ TailArgs<T> a) {
    pdl_wait();
    __shared__ double fs[kMaxDenseCells];
    __shared__ double mean;
    __shared__ TailLevel<T> Ls[kMaxTail];
    __shared__ const double* Msh;
    extern __shared__ __align__(16) unsigned char dyn[];
    const int n = a.n;
    if (threadIdx.x == 0) {
        for (int l = 0; l < n; ++l) Ls[l] = a.L[l];
        Msh = a.Minv;
        if (SMEM) {
            size_t off = 0;
            auto carve = [&](size_t bytes) {
                void* p = dyn + off;
                off += (bytes + 15) & ~(size_t)15;
                return p;
            };
            for (int l = 0; l < n; ++l) {
                TailLevel<T>& L = Ls[l];
                const int64_t cells = L.g.ncell();
                L.bx = (const T*)carve(sizeof(T) * L.g.nface(0));
                L.by = (const T*)carve(sizeof(T) * L.g.nface(1));
                L.bz = (const T*)carve(sizeof(T) * L.g.nface(2));
                if (USEW) L.w = (const T*)carve(sizeof(T) * cells);
                L.f = (T*)carve(sizeof(T) * cells);
                L.x = (T*)carve(sizeof(T) * cells);
            }
            const int64_t nc = Ls[n - 1].g.ncell();
            Msh = (const double*)carve(sizeof(double) * nc * nc);
        }
    }
    __syncthreads();
    if (SMEM) {
        // every thread issues its share of the copies as asynchronous global ->
        // shared copies and waits once, so the staging costs about one memory
        // latency instead of one per element a thread moves
        auto copy = [&](const T* src, const T* dst, int64_t cnt) {
            for (int64_t e = threadIdx.x; e < cnt; e += blockDim.x) async_copy(const_cast<T*>(dst) + e, src + e);
        };
        for (int l = 0; l < n; ++l) {
            const TailLevel<T>& G = a.L[l];
            const TailLevel<T>& L = Ls[l];
            copy(G.bx, L.bx, G.g.nface(0));
            copy(G.by, L.by, G.g.nface(1));
            copy(G.bz, L.bz, G.g.nface(2));
            if (USEW) copy(G.w, L.w, G.g.ncell());
        }
        copy(a.L[0].f, Ls[0].f, a.L[0].g.ncell());  // the other levels' f are restricted here
        const int64_t nc = a.L[n - 1].g.ncell();
        for (int64_t e = threadIdx.x; e < nc * nc; e += blockDim.x) async_copy(const_cast<double*>(Msh) + e, a.Minv + e);
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
    }
    for (int l = 0; l < n - 1; ++l) {
        const TailLevel<T> L = Ls[l];  // in registers: the loops below store through its pointers
        if (a.nu1 > 0) {
            tail_smooth<T, USEW>(L, a.nu1, true, false, a.omega);
        } else {
            const int cells = L.g.nx * L.g.ny * L.g.nz;
            for (int c = threadIdx.x; c < cells; c += blockDim.x) L.x[c] = T(0);
            __syncthreads();
        }
        tail_restrict<T>(L, Ls[l + 1]);
        __syncthreads();
    }
    tail_coarse_solve<T>(Ls[n - 1], Msh, fs, &mean);
    __syncthreads();
    for (int l = n - 2; l >= 0; --l) {
        tail_prolong<T>(Ls[l + 1], Ls[l]);
        __syncthreads();
        if (a.nu2 > 0) tail_smooth<T, USEW>(Ls[l], a.nu2, false, true, a.omega);
    }
    if (SMEM) {
        const int64_t cells = a.L[0].g.ncell();
        for (int64_t e = threadIdx.x; e < cells; e += blockDim.x) a.L[0].x[e] = Ls[0].x[e];
    }
}

// shared-memory bytes of the staged tail (16-byte aligned arrays)
template <typename T>
size_t tail_smem_bytes(const TailLevel<T>* levels, int n, bool use_w) {
    auto al = [](size_t b) { return (b + 15) & ~(size_t)15; };
    size_t b = 0;
    for (int l = 0; l < n; ++l) {
        const Geo& g = levels[l].g;
        b += al(sizeof(T) * g.nface(0)) + al(sizeof(T) * g.nface(1)) + al(sizeof(T) * g.nface(2));
        b += (use_w ? 3 : 2) * al(sizeof(T) * g.ncell());
    }
    const int64_t nc = levels[n - 1].g.ncell();
    return b + al(sizeof(double) * nc * nc);
}

}  // namespace

template <typename T>
void launch_tail_vcycle(const TailLevel<T>* levels, int n, const double* Minv, double omega, int nu1,
                        int nu2, bool use_w, cudaStream_t st) {
    TailArgs<T> a{};
    a.n = n;
    for (int l = 0; l < n; ++l) a.L[l] = levels[l];
    a.Minv = Minv;
    a.omega = (T)omega;
    a.nu1 = nu1;
    a.nu2 = nu2;
    // stage in shared memory when it fits (opt-in beyond 48 KB, once per variant)
    constexpr size_t kSmemMax = 200 * 1024;
    const size_t smem = tail_smem_bytes(levels, n, use_w);
    if (smem <= kSmemMax) {
        static bool opted[2] = {false, false};
        if (!opted[use_w ? 1 : 0]) {
            if (use_w)
                cudaFuncSetAttribute(tail_vcycle_kernel<T, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kSmemMax);
            else
                cudaFuncSetAttribute(tail_vcycle_kernel<T, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kSmemMax);
            opted[use_w ? 1 : 0] = true;
        }
        if (use_w)
            launch_pdl(tail_vcycle_kernel<T, true, true>, 1, kTailThreads, smem, st, a);
        else
            launch_pdl(tail_vcycle_kernel<T, false, true>, 1, kTailThreads, smem, st, a);
    } else if (use_w) {
        launch_pdl(tail_vcycle_kernel<T, true, false>, 1, kTailThreads, 0, st, a);
    } else {
        launch_pdl(tail_vcycle_kernel<T, false, false>, 1, kTailThreads, 0, st, a);
    }
    count_launch();
}

template void launch_tail_vcycle<float>(const TailLevel<float>*, int, const double*, double, int, int, bool,
                                        cudaStream_t);
template void launch_tail_vcycle<double>(const TailLevel<double>*, int, const double*, double, int, int,
                                         bool, cudaStream_t);

}  // namespace paris
