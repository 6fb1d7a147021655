// Host runtime of the projection library: context, multigrid level plan,
// workspace, the FP64 and mixed-precision Krylov drivers and the C ABI.
//
// Solver (Sec. 3.7 of the PARIS paper describes red-black SOR, Hypre's
// multigrid, an in-code V-cycle and a GPU Jacobi iteration; this library
// combines them as a preconditioner):
//   FP64  : conjugate gradients on A p = f (A = -L, f = -b, both mean-free)
//           preconditioned by one symmetric FP64 V-cycle (red-black SOR
//           smoother, 8-child averaging restriction, piecewise-constant
//           prolongation, rediscretised coarse coefficients, dense FP64 solve
//           on the coarsest grid).
//   MIXED : FP64 iterative refinement.  Each step computes the true residual
//           in FP64, solves A e = r approximately with flexible CG in FP32
//           preconditioned by the same V-cycle in FP32, and accumulates
//           p += e in FP64.  Dot products are summed across threads in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/paris.h"
#include "kernels.cuh"

using namespace paris;

namespace {

struct Level {
    Geo g;
    int fac[3] = {1, 1, 1};      // coarsening factor from the previous level
    double hrel[3] = {1, 1, 1};  // h_a of this level / h of level 0
    float* b32[3] = {nullptr, nullptr, nullptr};
    double* b64[3] = {nullptr, nullptr, nullptr};
    float* w32 = nullptr;
    double* w64 = nullptr;
    float* x32 = nullptr;
    float* f32 = nullptr;
    float* t32 = nullptr;  // Jacobi second buffer
    double* x64 = nullptr;
    double* f64 = nullptr;
    double* t64 = nullptr;
    double* sig64 = nullptr;  // diagonal excess of a Dirichlet-coupled operator (levels >= 1, on first use)
    float* sig32 = nullptr;   // its FP32 copy for the mixed form's V-cycle
    __half* b16[3] = {nullptr, nullptr, nullptr};  // level 1 of the mixed step: FP16 coefficients (see half1)
    float scale16 = 1.f;                           // their scale (the coefficient is b16 * scale16)
};

struct Alloc {
    std::vector<void*> ptrs;
    cudaError_t err = cudaSuccess;
    template <typename T>
    T* get(int64_t n) {
        if (err != cudaSuccess) return nullptr;
        void* p = nullptr;
        size_t bytes = (size_t)std::max<int64_t>(n, 1) * sizeof(T);
        err = cudaMalloc(&p, bytes);
        if (err != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return (T*)p;
    }
    void release() {
        for (void* p : ptrs) cudaFree(p);
        ptrs.clear();
    }
};

constexpr int kMaxDense = 128;
constexpr int kProfPool = 16384;  // event pairs per paris_profile(ctx, 1)

struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> ev;  // 2 per slot
    std::vector<int> slot_cls;
    std::vector<double> slot_bytes;
    std::vector<int> slot_n;  // launches bracketed by the slot's event pair
    int used = 0;
    int64_t launches[PARIS_K_COUNT] = {};
};

}  // namespace

struct paris_ctx {
    paris_grid grid;
    paris_opts opts;
    Geo g0;
    int64_t N = 0;
    cudaStream_t st = nullptr;
    std::vector<Level> lv;
    bool dense_coarse = false;
    Alloc mem;
    double* coarse_inv = nullptr;
    // FP64 Krylov vectors
    double *f = nullptr, *r = nullptr, *z = nullptr, *d = nullptr, *q = nullptr;
    // FP32 inner vectors
    float *r32 = nullptr, *z32 = nullptr, *d32 = nullptr, *q32 = nullptr, *e32 = nullptr;
    float* d32b = nullptr;  // the next direction of the fused direction update and product
    // level-0 FP32 coefficient copies (beta/h^2) and FP16 copies (beta) for
    // the V-cycle's finest-level passes
    float* b32_0[3] = {nullptr, nullptr, nullptr};
    __half* b16_0[3] = {nullptr, nullptr, nullptr};
    bool half0 = false;  // the current solve reads b16_0 in the level-0 V-cycle passes
    // FP32 half-densities rho/2 from which the finest level's FP32 kernels
    // rebuild their coefficients (paris_opts.level0_density)
    float* rh32 = nullptr;
    float2* rh2 = nullptr;  // rho/2 as (hi, lo) FP32 pairs for the refinement step
    __half* rh16 = nullptr;  // rho/2 in FP16 for the V-cycle's finest passes (paris_opts.level0_half_rho)
    bool half_rho = false;   // the current solve's V-cycle reads rh16, and level 1 its FP16 coefficients
    double rho_min = 1.0;    // the smaller density of the current projection step
    // plane order of the finest level's passes in the mixed form: each pass
    // starts where the one before it ended (its data still in L2), so
    // successive passes alternate; lz: the next one runs from the last plane
    bool lz = false;
    bool rho0 = false;  // the current solve's level-0 FP32 kernels read rh32 instead of b32_0
    // solid cells (Sec. 3.8): the caller's cell flags (1 fluid, 0 solid), or null
    const unsigned char* solid = nullptr;
    double n_fluid = 0.0;  // fluid cells (with solid set)
    // free-surface projections (Sec. 3.7.5; allocated on first use): the
    // finest level's diagonal excess and the cell classes; dirichlet: the
    // current solve's operator carries the excess (no null space)
    double* sig0 = nullptr;
    float* sig32_0 = nullptr;  // FP32 copy of sig0 times 1/h^2 (the mixed form's finest level)
    unsigned char* fs_cls = nullptr;
    unsigned char* fs_tmp = nullptr;
    bool dirichlet = false;
    // viscous-step multigrid work arrays (allocated on the first paris_viscous_solve_mg)
    HelmWork hmg{};
    std::vector<void*> hw_mem;
    double* partials = nullptr;
    Scal* scal = nullptr;
    Scal* scal_h = nullptr;  // pinned host mirror
    // projection-step scratch
    double* beta[3] = {nullptr, nullptr, nullptr};
    double* rhs = nullptr;
    // host-call staging (allocated on first use)
    double *hC = nullptr, *hu = nullptr, *hv = nullptr, *hw = nullptr, *hp = nullptr;
    bool mixed_ready = false;  // mixed_setup already ran for the current coefficients
    // host-buffer step: a copy stream and its ordering events (created on first use)
    cudaStream_t copy_st = nullptr;
    cudaEvent_t copy_ev[5] = {};
    cudaEvent_t scal_ev = nullptr;  // the host copy of scal of the inner loop's norms (read_scal_async)
    double last_mean_b = 0.0;
    Profiler prof;
    // CUDA graphs of the coarse part of the V-cycle (index 0: FP32, 1: FP64)
    cudaStream_t cap_stream = nullptr;
    bool cap_stream_broken = false;
    cudaGraphExec_t cg_exec[3] = {nullptr, nullptr, nullptr};
    int cg_kernels[3] = {0, 0, 0};
};

namespace {

#define CK(call)                                       \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) {                       \
            paris_internal_note_cuda_error(e_);        \
            return PARIS_ERR_CUDA;                     \
        }                                              \
    } while (0)

bool valid_grid(const paris_grid* g) {
    if (!g) return false;
    if (g->nx < 2 || g->ny < 2 || g->nz < 2) return false;
    if (!(g->h > 0.0) || !std::isfinite(g->h)) return false;
    for (int a = 0; a < 3; ++a)
        if (g->bc[a] != PARIS_PERIODIC && g->bc[a] != PARIS_WALL) return false;
    return true;
}

bool valid_opts(const paris_opts* o) {
    if (!o) return false;
    if (!(o->tol > 0.0) || o->max_iter < 1) return false;
    if (o->precision != PARIS_FP64 && o->precision != PARIS_MIXED) return false;
    if (o->nu1 < 0 || o->nu2 < 0 || o->nu1 + o->nu2 < 1 || o->nu1 > 16 || o->nu2 > 16) return false;
    if (!(o->omega > 0.0 && o->omega < 2.0)) return false;
    if (o->smoother < PARIS_SMOOTH_RBGS || o->smoother > PARIS_SMOOTH_RBGS_2PASS) return false;
    if (o->coarse_max_cells < 1 || o->coarse_max_cells > kMaxDense) return false;
    if (!(o->inner_tol > 0.0 && o->inner_tol < 1.0)) return false;
    if (o->slab_planes < 0) return false;
    if (o->level0_density != 0 && o->level0_density != 1) return false;
    if (o->level0_tiles < 0 || o->level0_tiles > 2) return false;
    if (o->level0_half_rho != 0 && o->level0_half_rho != 1) return false;
    if (o->coarse_tail != 0 && o->coarse_tail != 1) return false;
    return true;
}

// Level plan: halve every axis while all are even and >= 4; once that stops,
// halve the axes that still can (semi-coarsening) while the level has more
// than coarse_max_cells cells.  The paper's in-code multigrid (Sec. 3.7.3)
// needs 2^n points per direction; this plan also covers sizes such as 48 or 96.
std::vector<Level> plan_levels(const paris_grid& gr, int coarse_max) {
    std::vector<Level> out;
    Level l0;
    l0.g = Geo{gr.nx, gr.ny, gr.nz, gr.bc[0] == PARIS_WALL, gr.bc[1] == PARIS_WALL,
               gr.bc[2] == PARIS_WALL};
    out.push_back(l0);
    for (;;) {
        const Level& c = out.back();
        if (c.g.ncell() <= coarse_max) break;
        int n[3] = {c.g.nx, c.g.ny, c.g.nz};
        bool can[3];
        bool all = true, any = false;
        for (int a = 0; a < 3; ++a) {
            can[a] = (n[a] % 2 == 0) && n[a] >= 4;
            all = all && can[a];
            any = any || can[a];
        }
        if (!any) break;
        Level nl;
        nl.g = c.g;
        for (int a = 0; a < 3; ++a) {
            int f = (all || can[a]) ? 2 : 1;
            nl.fac[a] = f;
            nl.hrel[a] = c.hrel[a] * f;
            n[a] /= f;
        }
        nl.g.nx = n[0];
        nl.g.ny = n[1];
        nl.g.nz = n[2];
        out.push_back(nl);
    }
    return out;
}

paris_status alloc_ctx(paris_ctx* c) {
    Alloc& m = c->mem;
    const int64_t N = c->N;
    c->lv = plan_levels(c->grid, c->opts.coarse_max_cells);
    const Level& last = c->lv.back();
    c->dense_coarse = last.g.ncell() <= kMaxDense;
    for (size_t l = 0; l < c->lv.size(); ++l) {
        Level& L = c->lv[l];
        const int64_t n = L.g.ncell();
        if (l > 0) {
            for (int a = 0; a < 3; ++a) {
                L.b32[a] = m.get<float>(L.g.nface(a));
                L.b64[a] = m.get<double>(L.g.nface(a));
            }
            L.x32 = m.get<float>(n);
            L.f32 = m.get<float>(n);
            L.x64 = m.get<double>(n);
            L.f64 = m.get<double>(n);
        }
        L.w32 = m.get<float>(n);
        L.w64 = m.get<double>(n);
        L.t32 = m.get<float>(n);
        L.t64 = m.get<double>(n);
    }
    if (c->dense_coarse) c->coarse_inv = m.get<double>(last.g.ncell() * last.g.ncell());
    c->f = m.get<double>(N);
    c->r = m.get<double>(N);
    c->z = m.get<double>(N);
    c->d = m.get<double>(N);
    c->q = m.get<double>(N);
    c->r32 = m.get<float>(N);
    c->z32 = m.get<float>(N);
    c->d32 = m.get<float>(N);
    c->q32 = m.get<float>(N);
    c->e32 = m.get<float>(N);
    if (rho0_fits(c->g0)) c->d32b = m.get<float>(N);
    for (int a = 0; a < 3; ++a) {
        c->b32_0[a] = m.get<float>(c->g0.nface(a));
        c->b16_0[a] = m.get<__half>(c->g0.nface(a));
        c->beta[a] = m.get<double>(c->g0.nface(a));
    }
    c->rhs = m.get<double>(N);
    if (rho0_fits(c->g0)) {
        c->rh32 = m.get<float>(N);
        c->rh2 = m.get<float2>(N);
        c->rh16 = m.get<__half>(N);
        if (c->lv.size() > 1)
            for (int a = 0; a < 3; ++a) c->lv[1].b16[a] = m.get<__half>(c->lv[1].g.nface(a));
    }
    // block partials: up to 4 values per block of the largest reducing grid
    c->partials = m.get<double>(std::max(max_reduce_blocks(c->g0), rho0_matvec_blocks(c->g0)) * 4);
    c->scal = m.get<Scal>(1);
    if (m.err != cudaSuccess) return m.err == cudaErrorMemoryAllocation ? PARIS_ERR_NO_MEMORY : PARIS_ERR_CUDA;
    if (cudaMallocHost(&c->scal_h, sizeof(Scal)) != cudaSuccess) return PARIS_ERR_NO_MEMORY;
    CK(cudaMemsetAsync(c->scal, 0, sizeof(Scal), c->st));
    return PARIS_OK;
}

void drop_graphs(paris_ctx* c) {
    for (auto& g : c->cg_exec)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

paris_status read_scal(paris_ctx* c) {
    CK(cudaMemcpyAsync(c->scal_h, c->scal, sizeof(Scal), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (c->scal_h->wait_fail) {  // a staged kernel's bounded wait gave up: clear the word, report it
        CK(cudaMemsetAsync(&c->scal->wait_fail, 0, sizeof(unsigned), c->st));
        return PARIS_ERR_TIMEOUT;
    }
    return PARIS_OK;
}

// read_scal in two halves: the copy queued (and an event after it), so that
// more work can be queued behind it, then the wait for that copy only
paris_status read_scal_async(paris_ctx* c) {
    if (!c->scal_ev) CK(cudaEventCreateWithFlags(&c->scal_ev, cudaEventDisableTiming));
    CK(cudaMemcpyAsync(c->scal_h, c->scal, sizeof(Scal), cudaMemcpyDeviceToHost, c->st));
    CK(cudaEventRecord(c->scal_ev, c->st));
    return PARIS_OK;
}
paris_status read_scal_wait(paris_ctx* c) {
    CK(cudaEventSynchronize(c->scal_ev));
    if (c->scal_h->wait_fail) {
        CK(cudaMemsetAsync(&c->scal->wait_fail, 0, sizeof(unsigned), c->st));
        return PARIS_ERR_TIMEOUT;
    }
    return PARIS_OK;
}

// Brackets one launch of an instrumented kernel class with an event pair
// when profiling is on (see paris_profile).
struct ProfScope {
    paris_ctx* c;
    int slot = -1;
    // n: the launches the pair brackets (consecutive launches of one class
    // share a pair, so that the pair's own cost is spread over them)
    ProfScope(paris_ctx* c_, int cls, double bytes, int n = 1) : c(c_) {
        Profiler& P = c->prof;
        if (!P.on || cls < 0) return;
        P.launches[cls] += n;
        if (P.used < kProfPool) {
            slot = P.used++;
            P.slot_cls[slot] = cls;
            P.slot_bytes[slot] = bytes;
            P.slot_n[slot] = n;
            cudaEventRecord(P.ev[2 * slot], c->st);
        }
    }
    ~ProfScope() {
        if (slot >= 0) cudaEventRecord(c->prof.ev[2 * slot + 1], c->st);
    }
};

double beta_count(const Geo& g) { return (double)(g.nface(0) + g.nface(1) + g.nface(2)); }

// ------------------------------------------------------------- V-cycle ---

template <typename T>
struct Prec;
template <>
struct Prec<float> {
    static float* b(Level& L, int a) { return L.b32[a]; }
    static float* w(Level& L) { return L.w32; }
    static float* x(Level& L) { return L.x32; }
    static float* f(Level& L) { return L.f32; }
    static float* t(Level& L) { return L.t32; }
    static float* sig(Level& L) { return L.sig32; }
};
template <>
struct Prec<double> {
    static double* b(Level& L, int a) { return L.b64[a]; }
    static double* w(Level& L) { return L.w64; }
    static double* x(Level& L) { return L.x64; }
    static double* f(Level& L) { return L.f64; }
    static double* t(Level& L) { return L.t64; }
    static double* sig(Level& L) { return L.sig64; }
};

template <typename T>
Coef<T> level_coef(paris_ctx* c, int l, const Coef<T>& c0) {
    if (l == 0) return c0;
    Level& L = c->lv[l];
    Coef<T> cf{Prec<T>::b(L, 0), Prec<T>::b(L, 1), Prec<T>::b(L, 2), T(1)};
    if (c->dirichlet) cf.sig = Prec<T>::sig(L);
    return cf;
}

int tail_start(const paris_ctx* c);

// Per-solve set-up of the hierarchy in precision T: coarse coefficients,
// inverse diagonals, dense coarsest inverse.
template <typename T>
void setup_hierarchy(paris_ctx* c, const Coef<T>& c0) {
    const int nl = (int)c->lv.size();
    for (int l = 1; l < nl; ++l) {
        Level& L = c->lv[l];
        Level& F = c->lv[l - 1];
        Coef<T> cf = level_coef<T>(c, l - 1, c0);
        double ratio2[3];
        for (int a = 0; a < 3; ++a) ratio2[a] = (double)L.fac[a] * L.fac[a];
        T* out[3] = {Prec<T>::b(L, 0), Prec<T>::b(L, 1), Prec<T>::b(L, 2)};
        if constexpr (sizeof(T) == 4) {
            if (l == 1 && c->rho0) {
                // with the FP16 rho/2 of the V-cycle, level 1 gets FP16 coefficients too: the
                // sums of four fine faces' 1/(rh_L + rh_R) times a power of two s16 that puts
                // them below 2^14 (all between 2^14 rho_min/rho_max / 2 and 2^14)
                float s16 = 1.f;
                if (c->half_rho) {
                    s16 = std::ldexp(1.0f, (int)std::floor(std::log2(4096.0 * c->rho_min)));
                    L.scale16 = (float)(1.0 / (16.0 * c->grid.h * c->grid.h * (double)s16));
                }
                launch_coarse_beta_rho(F.g, c->rh32, c->grid.h, L.g, out, c->st, c->half_rho ? L.b16 : nullptr, s16);
                continue;
            }
        }
        launch_coarse_beta<T>(F.g, cf, L.g, L.fac, ratio2, out, c->st);
        if (c->dirichlet) launch_coarse_sig<T>(F.g, cf.sig, (double)cf.scale, L.g, L.fac, Prec<T>::sig(L), c->st);
    }
    // inverse diagonals: read by the FP64 smoothers, by Jacobi, by the tail
    // launch and by every smoother of an operator with a diagonal excess; the
    // other FP32 red-black sweeps recompute them from the coefficients they
    // load (the same value)
    const int t = tail_start(c);
    if (sizeof(T) == 8 || c->opts.smoother == PARIS_SMOOTH_JACOBI || c->dirichlet) {
        for (int l = 0; l < nl; ++l)
            launch_inv_diag<T>(c->lv[l].g, level_coef<T>(c, l, c0), Prec<T>::w(c->lv[l]), c->st);
    } else if (t > 0) {
        for (int l = t; l < nl; ++l)
            launch_inv_diag<T>(c->lv[l].g, level_coef<T>(c, l, c0), Prec<T>::w(c->lv[l]), c->st);
    }
    if (c->dense_coarse)
        launch_coarse_inverse<T>(c->lv[nl - 1].g, level_coef<T>(c, nl - 1, c0), c->coarse_inv, c->st);
}

#ifndef PARIS_ZREV
#define PARIS_ZREV 1
#endif
constexpr bool kZrev = PARIS_ZREV != 0;

// the plane order of the next finest-level pass of the mixed form (see
// paris_ctx::lz), and the order of the one after it
bool take_dir(paris_ctx* c) {
    const bool r = kZrev && c->lz;
    c->lz = !c->lz;
    return r;
}

template <typename T>
void smooth(paris_ctx* c, int l, const Coef<T>& cf, const T* f, T* x, int sweeps, bool first_zero,
            bool reverse) {
    Level& L = c->lv[l];
    const paris_opts& o = c->opts;
    const double n = (double)L.g.ncell(), sz = sizeof(T), nb = beta_count(L.g);
    const int cls = l == 0 ? PARIS_K_SMOOTH0 : -1;
    // FP64: a division costs more than reading 1/D; a diagonal excess is only in 1/D
    const bool use_w = sizeof(T) == 8 || cf.sig != nullptr;
    if (o.smoother == PARIS_SMOOTH_RBGS_2PASS ||
        (o.smoother == PARIS_SMOOTH_RBGS && !rbgs_fused_fits(L.g))) {
        // Large levels run each colour pass slab by slab: the second colour of
        // slab s follows the first colour of slab s+1, while slab s is still
        // in L2, so a sweep reads the level from HBM about once instead of
        // twice.  The last slab's first colour runs early because with a
        // periodic z axis it needs plane 0's second colour not yet updated.
        // Every cell sees the same values as in two full passes.
        const int nz = L.g.nz;
        const int S = o.slab_planes > 0 ? o.slab_planes : nz;
        const int m = (nz + S - 1) / S;
        const bool slabs = o.slab_planes > 0 && m >= 4;
        // the finest level's passes of this smoothing phase run back to back:
        // one event pair brackets all of them (their bytes and launch count
        // summed), so that the pair's own cost is spread over the phase
        int phase_cls = -1;
        double phase_bytes = 0.0;
        int phase_n = 0;
        if (cls >= 0) {
            // bytes per pass: x at every cell (neighbours and the updated colour),
            // f and the write of the updated colour, plus the coefficients
            // (three face arrays, or rho/2 once, 4 or 2 bytes a cell); a
            // zero-initial pass reads no x and writes both colours (plane-tile
            // zero pass: the updated colour only, and the pass after it reads
            // neither colour's old value of its own cells)
            for (int s = 0; s < sweeps; ++s) {
                const bool z0 = first_zero && s == 0;
                const bool v0 = sizeof(T) == 4 && l == 0 && c->rho0;
                const bool h16 = sizeof(T) == 4 && l == 0 && c->half0;
                const double bsz = h16 ? 2.0 : (double)sz;
                const bool tile0 = v0 && rho0_tile_pass(L.g, o.level0_tiles);
                const double rhb = c->half_rho ? 2.0 : 4.0;  // bytes of rho/2 per cell
                phase_bytes += v0 ? (z0 ? (tile0 ? 1.0 : 1.5) : 2.0) * n * sz + rhb * n
                                  : (z0 ? 2 * n * sz : 2.5 * n * sz + nb * bsz);
                phase_bytes += v0 ? ((z0 && tile0) ? 1.5 : 2.0) * n * sz + rhb * n : 2.5 * n * sz + nb * bsz;
                phase_n += slabs ? 2 * m : 2;
            }
            phase_cls = cls;
        }
        ProfScope phase(c, phase_cls, phase_bytes, phase_n);
        for (int s = 0; s < sweeps; ++s) {
            const bool z0 = first_zero && s == 0;
            const int c0 = reverse ? 1 : 0;
            // FP32 solve, finest level: coefficients from the FP16 copies or
            // rebuilt from the cell densities
            const bool h16 = sizeof(T) == 4 && l == 0 && c->half0;
            const bool v0 = sizeof(T) == 4 && l == 0 && c->rho0;
            const double bsz = h16 ? 2.0 : (double)sz;
            auto pass = [&](int color, bool zero, int a, int b) {
                if constexpr (sizeof(T) == 4) {
                    if (v0) {
                        // after a zero pass the other colour is still unwritten on the
                        // plane-tile path: the second pass of that sweep takes it as zero
                        // successive passes alternate their plane order, each starting
                        // where the previous one ended (planes still in L2)
                        launch_rbgs_rho(L.g, c->rh32, c->grid.h, (const float*)f, (float*)x, color, o.omega,
                                        zero, c->st, a, b, o.level0_tiles, z0 && !zero, &c->scal->wait_fail,
                                        c->half_rho ? c->rh16 : nullptr, take_dir(c));
                        return;
                    }
                    if (h16) {
                        // FP16 arrays hold beta itself: scale by 1/h^2 in the kernel
                        launch_rbgs_h(L.g, c->b16_0, (float)(1.0 / (c->grid.h * c->grid.h)), f, x, color,
                                      o.omega, zero, c->st, a, b);
                        return;
                    }
                    if (l == 1 && c->rho0 && c->half_rho) {  // level 1 of the mixed step: FP16 coefficients
                        launch_rbgs_h(L.g, L.b16, L.scale16, f, x, color, o.omega, zero, c->st, a, b);
                        return;
                    }
                }
                launch_rbgs<T>(L.g, cf, Prec<T>::w(L), f, x, color, o.omega, zero, c->st, a, b);
            };
            auto first = [&](int a, int b) { pass(c0, z0, a, b); };
            auto second = [&](int a, int b) { pass(1 - c0, false, a, b); };
            if (!slabs) {
                first(0, nz);
                second(0, nz);
                continue;
            }
            auto lo = [&](int q) { return q * S; };
            auto hi = [&](int q) { return std::min(nz, (q + 1) * S); };
            first(lo(0), hi(0));
            first(lo(m - 1), hi(m - 1));
            for (int q = 1; q <= m - 2; ++q) {
                first(lo(q), hi(q));
                second(lo(q - 1), hi(q - 1));
            }
            second(lo(m - 2), hi(m - 2));
            second(lo(m - 1), hi(m - 1));
        }
        return;
    }
    // ping-pong between x and the level's second buffer, ending in x
    T* bufs[2] = {x, Prec<T>::t(L)};
    int cur = 0;
    for (int s = 0; s < sweeps; ++s) {
        const bool z0 = first_zero && s == 0;
        const int remaining = sweeps - s;
        const int out = z0 ? ((remaining % 2 == 1) ? 0 : 1) : 1 - cur;
        const T* in = z0 ? nullptr : bufs[cur];
        if (o.smoother == PARIS_SMOOTH_JACOBI) {
            ProfScope ps(c, cls, (z0 ? 3 * n : 4 * n + nb) * sz);
            launch_jacobi<T>(L.g, cf, Prec<T>::w(L), f, in ? in : f, bufs[out], o.omega, z0, c->st);
        } else {
            ProfScope ps(c, cls, ((z0 ? 2 * n : 3 * n) + nb + (use_w ? n : 0)) * sz);
            launch_rbgs_fused<T>(L.g, cf, Prec<T>::w(L), f, in, bufs[out], reverse ? 1 : 0, o.omega, z0,
                                 use_w, c->st);
        }
        cur = out;
    }
    if (cur != 0)
        cudaMemcpyAsync(x, bufs[cur], sizeof(T) * L.g.ncell(), cudaMemcpyDeviceToDevice, c->st);
}

// Pre-smoothing on level l and restriction of its residual to level l+1.
template <typename T>
void vdown(paris_ctx* c, const Coef<T>& c0, const T* f0, T* x0, int l) {
    const paris_opts& o = c->opts;
    const T* f = l == 0 ? f0 : Prec<T>::f(c->lv[l]);
    T* x = l == 0 ? x0 : Prec<T>::x(c->lv[l]);
    Coef<T> cf = level_coef<T>(c, l, c0);
    if (o.nu1 > 0) smooth<T>(c, l, cf, f, x, o.nu1, true, false);
    else cudaMemsetAsync(x, 0, sizeof(T) * c->lv[l].g.ncell(), c->st);
    Level& C = c->lv[l + 1];
    const double n = (double)c->lv[l].g.ncell();
    const bool h16 = sizeof(T) == 4 && l == 0 && c->half0;
    const bool v0 = sizeof(T) == 4 && l == 0 && c->rho0;
    ProfScope ps(c, l == 0 ? PARIS_K_RESTRICT0 : -1,
                 (2 * n + (double)C.g.ncell()) * sizeof(T) +
                     (v0 ? n * (c->half_rho ? 2.0 : (double)sizeof(T)) : beta_count(c->lv[l].g) * (h16 ? 2 : sizeof(T))));
    if constexpr (sizeof(T) == 4) {
        if (v0) {
            launch_restrict_rho(c->lv[l].g, c->rh32, c->grid.h, (const float*)f, (const float*)x, C.g,
                                (float*)Prec<T>::f(C), c->st, c->opts.level0_tiles != 0,
                                c->half_rho ? c->rh16 : nullptr, take_dir(c));
            return;
        }
        if (h16) {
            launch_restrict_residual_h(c->lv[l].g, c->b16_0, (float)(1.0 / (c->grid.h * c->grid.h)), f, x, C.g,
                                       C.fac, Prec<T>::f(C), c->st);
            return;
        }
        if (l == 1 && c->rho0 && c->half_rho) {
            const Level& L1 = c->lv[1];
            launch_restrict_residual_h(L1.g, L1.b16, L1.scale16, f, x, C.g, C.fac, Prec<T>::f(C), c->st);
            return;
        }
    }
    launch_restrict_residual<T>(c->lv[l].g, cf, f, x, C.g, C.fac, Prec<T>::f(C), c->st);
}

// Exact (dense) or smoothed solve on the coarsest level.
template <typename T>
void vcoarse(paris_ctx* c, const Coef<T>& c0, const T* f0, T* x0) {
    const int nl = (int)c->lv.size();
    Level& C = c->lv[nl - 1];
    const T* f = nl == 1 ? f0 : Prec<T>::f(C);
    T* x = nl == 1 ? x0 : Prec<T>::x(C);
    if (c->dense_coarse) {
        launch_coarse_solve<T>(C.g, c->coarse_inv, f, x, c->st, c->dirichlet);
    } else {
        Coef<T> cf = level_coef<T>(c, nl - 1, c0);
        smooth<T>(c, nl - 1, cf, f, x, 8, true, false);
        smooth<T>(c, nl - 1, cf, f, x, 8, false, true);
    }
}

// Prolongation from level l+1 onto level l and post-smoothing on level l.
template <typename T>
void vup(paris_ctx* c, const Coef<T>& c0, const T* f0, T* x0, int l) {
    const paris_opts& o = c->opts;
    const T* f = l == 0 ? f0 : Prec<T>::f(c->lv[l]);
    T* x = l == 0 ? x0 : Prec<T>::x(c->lv[l]);
    Coef<T> cf = level_coef<T>(c, l, c0);
    Level& C = c->lv[l + 1];
    {
        const double n = (double)c->lv[l].g.ncell();
        ProfScope ps(c, l == 0 ? PARIS_K_PROLONG0 : -1, (2 * n + (double)C.g.ncell()) * sizeof(T));
        bool split = false;
        if constexpr (sizeof(T) == 4) {
            if (l == 0 && c->rho0) {
                launch_prolong_split(c->lv[l].g, C.g, (const float*)Prec<T>::x(C), (float*)x, c->st, take_dir(c));
                split = true;
            }
        }
        if (!split) launch_prolong_add<T>(c->lv[l].g, C.g, C.fac, Prec<T>::x(C), x, c->st);
    }
    if (o.nu2 > 0) smooth<T>(c, l, cf, f, x, o.nu2, false, true);
}

// Levels with at most this many cells, down to the dense coarsest level,
// run as one single-block launch (launch_tail_vcycle).
#ifndef PARIS_TAIL_CELLS
#define PARIS_TAIL_CELLS 4096
#endif
constexpr int64_t kTailCells = PARIS_TAIL_CELLS;

// First level of that tail, or -1 (the tail needs the two-pass red-black
// smoother, a dense coarsest level and at least one level above it).
int tail_start(const paris_ctx* c) {
    const int nl = (int)c->lv.size();
    if (c->opts.coarse_tail == 0 || !c->dense_coarse || c->opts.smoother != PARIS_SMOOTH_RBGS_2PASS || nl < 3 ||
        c->dirichlet)
        return -1;
    // level 1 with FP16 coefficients (the mixed step's FP16 rho/2) keeps its own kernels
    const int lo = (c->rho0 && c->half_rho) ? 2 : 1;
    int t = nl - 1;
    while (t - 1 >= lo && c->lv[t - 1].g.ncell() <= kTailCells) --t;
    if (t >= nl - 1 || nl - t > kMaxTail) return -1;
    return t;
}

template <typename T>
void launch_tail(paris_ctx* c, int t) {
    const int nl = (int)c->lv.size();
    TailLevel<T> tl[kMaxTail];
    for (int l = t; l < nl; ++l) {
        Level& L = c->lv[l];
        TailLevel<T>& d = tl[l - t];
        d.g = L.g;
        for (int a = 0; a < 3; ++a) d.fac[a] = L.fac[a];
        // multipliers of the index divisions (ceil(2^32 / n); n = 1 is special-cased in the kernel)
        auto mul = [](int n) { return n > 1 ? (unsigned)((0x100000000ull + (unsigned)n - 1) / (unsigned)n) : 0u; };
        d.mx = mul(L.g.nx);
        d.my = mul(L.g.ny);
        d.mp = mul((L.g.nx + 1) / 2);
        d.scale = T(1);
        d.bx = Prec<T>::b(L, 0);
        d.by = Prec<T>::b(L, 1);
        d.bz = Prec<T>::b(L, 2);
        d.w = Prec<T>::w(L);  // the inverse diagonals (set up with the hierarchy)
        d.x = Prec<T>::x(L);
        d.f = Prec<T>::f(L);
    }
    launch_tail_vcycle<T>(tl, nl - t, c->coarse_inv, c->opts.omega, c->opts.nu1, c->opts.nu2, true, c->st);
}

// Levels 1 .. L-1 of the V-cycle (level 0's restriction already done).
template <typename T>
void coarse_part(paris_ctx* c, const Coef<T>& c0) {
    const int nl = (int)c->lv.size();
    const int t = tail_start(c);
    if (t > 0) {
        for (int l = 1; l < t; ++l) vdown<T>(c, c0, nullptr, nullptr, l);
        launch_tail<T>(c, t);
        for (int l = t - 1; l >= 1; --l) vup<T>(c, c0, nullptr, nullptr, l);
        return;
    }
    for (int l = 1; l < nl - 1; ++l) vdown<T>(c, c0, nullptr, nullptr, l);
    vcoarse<T>(c, c0, nullptr, nullptr);
    for (int l = nl - 2; l >= 1; --l) vup<T>(c, c0, nullptr, nullptr, l);
}

// The part of the V-cycle below level 0 (levels 1 .. L-1) only reads and
// writes the context's own level arrays, so it is captured once per
// precision into a CUDA graph and replayed: dozens of small launches on the
// coarse levels become one graph launch.  Captured on the context's private
// stream (the legacy default stream cannot be captured), launched on the
// context's stream.
template <typename T>
bool coarse_graph_launch(paris_ctx* c, const Coef<T>& c0) {
    const int nl = (int)c->lv.size();
    // FP32 graphs with level 1 from the FP32 or from the FP16 coefficients, FP64
    const int slot = sizeof(T) == 8 ? 1 : ((c->rho0 && c->half_rho) ? 2 : 0);
    if (nl < 3 || !c->cap_stream) return false;
    if (!c->cg_exec[slot]) {
        cudaStream_t user = c->st;
        c->st = c->cap_stream;
        const long long before = launch_count();
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            coarse_part<T>(c, c0);
            e = cudaStreamEndCapture(c->st, &g);
        }
        c->st = user;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->cg_exec[slot], g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->cg_exec[slot] = nullptr;
            c->cap_stream_broken = true;  // fall back to direct launches
            return false;
        }
        c->cg_kernels[slot] = (int)(launch_count() - before);
        count_launch(-c->cg_kernels[slot]);  // counted when replayed instead
    }
    if (cudaGraphLaunch(c->cg_exec[slot], c->st) != cudaSuccess) return false;
    count_launch(c->cg_kernels[slot]);
    return true;
}

// x0 = V(f0): one symmetric V-cycle for A x = f on level 0 (x0 overwritten).
template <typename T>
void vcycle(paris_ctx* c, const Coef<T>& c0, const T* f0, T* x0) {
    const int nl = (int)c->lv.size();
    if (nl >= 3 && !c->cap_stream_broken && !c->dirichlet) {
        vdown<T>(c, c0, f0, x0, 0);
        {
            ProfScope ps(c, PARIS_K_COARSE, 0.0);
            if (!coarse_graph_launch<T>(c, c0)) coarse_part<T>(c, c0);
        }
        vup<T>(c, c0, f0, x0, 0);
        return;
    } else {
        for (int l = 0; l < nl - 1; ++l) vdown<T>(c, c0, f0, x0, l);
    }
    vcoarse<T>(c, c0, f0, x0);
    for (int l = nl - 2; l >= 0; --l) vup<T>(c, c0, f0, x0, l);
}

// ------------------------------------------------------------- drivers ---

struct SolveOut {
    int iters = 0, outer = 0;
    bool converged = false, nonfinite = false;
};

bool meets(const paris_ctx* c, const Scal& s) {
    const double t = c->opts.tol;
    return s.rr <= t * t * s.bnorm2 && s.rinf <= t * s.binf;
}

// Common prologue: mean of rhs (unless the caller already left it in
// scal->mean_b), f = -(rhs - mean), norms of f and max |x0| of the initial guess.
paris_status prologue(paris_ctx* c, const double* rhs, const double* x0, bool mean_known) {
    int64_t nb;
    if (!mean_known) {
        if (c->solid) {  // the mean over the fluid cells (the masked operator's constant mode)
            launch_fluid_mean(c->N, c->solid, rhs, c->partials, c->scal, c->st);
        } else {
            nb = launch_sum(c->N, rhs, c->partials, c->st);
            finalize(c->partials, nb, 3, 2, c->scal, FIN_MEAN_B, (double)c->N, c->st);
        }
    }
    launch_make_rhs(c->N, rhs, c->scal, c->f, x0, c->partials, c->st, FinSpec{c->scal, 4, 0xA, FIN_BNORMS, 0.0},
                    c->solid);
    CK(cudaGetLastError());
    return PARIS_OK;
}

// r = f - A x in FP64 (r32: the scaled FP32 copy only); zero_ok: x is still
// the initial guess the prologue measured.
paris_status true_residual(paris_ctx* c, const Coef<double>& c64, const double* x, float* r32,
                           bool zero_ok = false, bool keep_r64 = false) {
    if (r32) finalize(c->partials, 0, 1, 0, c->scal, FIN_SCALE, 0.0, c->st);
    {
        const double n = (double)c->N;
        ProfScope ps(c, PARIS_K_RESID64, (16 * n + 8 * beta_count(c->g0)) + (r32 ? 4 : 8) * n);
        launch_residual64(c->g0, c64, c->f, x, (r32 && !keep_r64) ? nullptr : c->r, r32, c->scal, c->partials,
                          zero_ok, c->st, FinSpec{c->scal, 3, 2, FIN_RNORMS, 0.0}, r32 && c->rho0);
    }
    ProfScope ps(c, PARIS_K_KRYLOV, 0.0);
    CK(cudaGetLastError());
    return read_scal(c);
}

// FP64 multigrid-preconditioned CG from the initial guess in x.
paris_status solve_fp64(paris_ctx* c, const Coef<double>& c64, double* x, SolveOut& out,
                        int max_iter, bool fresh) {
    {
        ProfScope ps(c, PARIS_K_SETUP, 0.0);
        setup_hierarchy<double>(c, c64);
    }
    paris_status s = true_residual(c, c64, x, nullptr, fresh);  // r = f - A x
    if (s != PARIS_OK) return s;
    if (c->scal_h->nonfinite > 0) { out.nonfinite = true; return PARIS_OK; }
    if (c->scal_h->bnorm2 == 0.0 || meets(c, *c->scal_h)) { out.converged = true; return PARIS_OK; }
    const int64_t N = c->N;
    int restarts = 0;
    while (out.iters < max_iter) {
        vcycle<double>(c, c64, c->r, c->z);
        {
            ProfScope ps(c, PARIS_K_KRYLOV, 0.0);
            launch_dot2<double>(N, c->r, c->z, nullptr, c->partials, c->st,
                                FinSpec{c->scal, 2, 0, FIN_RHO_INIT, 0.0});
            std::swap(c->d, c->z);  // first direction d = z: exchange the buffers
        }
        bool conv = false;
        while (out.iters < max_iter) {
            {
                ProfScope ps(c, PARIS_K_MATVEC0, (2.0 * N + beta_count(c->g0)) * 8);
                launch_matvec_dot<double>(c->g0, c64, c->d, c->q, c->partials, c->st,
                                          FinSpec{c->scal, 1, 0, FIN_ALPHA, 0.0});
            }
            {
                ProfScope ps(c, PARIS_K_KRYLOV, 0.0);
                launch_update_xr<double>(N, c->scal, c->d, c->q, x, c->r, c->partials, c->st,
                                         FinSpec{c->scal, 3, 2, FIN_RNORMS, 0.0});
                s = read_scal(c);
            }
            ++out.iters;
            if (s != PARIS_OK) return s;
            if (c->scal_h->nonfinite > 0) { out.nonfinite = true; return PARIS_OK; }
            if (meets(c, *c->scal_h)) { conv = true; break; }
            vcycle<double>(c, c64, c->r, c->z);
            ProfScope ps(c, PARIS_K_KRYLOV, 0.0);
            launch_dot2<double>(N, c->r, c->z, nullptr, c->partials, c->st,
                                FinSpec{c->scal, 2, 0, FIN_RHO_BETA, 0.0});
            launch_xpby<double>(N, c->scal, c->z, c->d, c->st);
        }
        // verify with the true residual; restart from it if the recurrence drifted
        s = true_residual(c, c64, x, nullptr);
        if (s != PARIS_OK) return s;
        if (meets(c, *c->scal_h)) { out.converged = true; return PARIS_OK; }
        if (!conv || ++restarts > 3) return PARIS_OK;
    }
    return PARIS_OK;
}

// Mixed precision: FP64 iterative refinement around FP32 flexible CG.
// The level-0 FP32 kernels can rebuild their coefficients from the cell
// densities (paris_opts.level0_density) when the grid and the smoother allow it.
bool rho0_usable(const paris_ctx* c) {
    const paris_opts& o = c->opts;
    if (!o.level0_density || o.precision != PARIS_MIXED || o.smoother != PARIS_SMOOTH_RBGS_2PASS ||
        o.half_coefficients || !c->rh32 || !c->rh2 || c->lv.size() < 3 || c->solid)
        return false;
    const Level& L1 = c->lv[1];
    return L1.fac[0] == 2 && L1.fac[1] == 2 && L1.fac[2] == 2;
}

// Clears the per-solve level-0 mode flags on every exit path.
struct Level0Mode {
    paris_ctx* c;
    ~Level0Mode() {
        c->rho0 = false;
        c->half0 = false;
        c->half_rho = false;
    }
};

// The set-up of the mixed solve: FP32 copies of the finest coefficients (or
// nothing, with the finest level from rho/2) and the FP32 hierarchy.  It
// depends on the coefficients only, so the projection step runs it before
// the right-hand side and the initial guess are needed (mixed_ready).
void mixed_setup(paris_ctx* c, const Coef<double>& c64, bool rho0) {
    const double ih2 = 1.0 / (c->grid.h * c->grid.h);
    const double* b64[3] = {c64.bx, c64.by, c64.bz};
    c->rho0 = rho0;
    c->half0 = !rho0 && c->opts.half_coefficients != 0 && !c->dirichlet;
    Coef<float> c32{c->b32_0[0], c->b32_0[1], c->b32_0[2], 1.0f};
    ProfScope ps(c, PARIS_K_SETUP, 0.0);
    if (!rho0) {
        launch_convert_beta<float>(c->g0, b64, ih2, c->b32_0, c->st);
        if (c->half0) launch_convert_beta_half(c->g0, b64, c->b16_0, c->st);
    }
    if (c->dirichlet) {  // the diagonal excess, scaled like the FP32 coefficients
        launch_convert_scaled(c->N, c64.sig, ih2, c->sig32_0, c->st);
        c32.sig = c->sig32_0;
    }
    setup_hierarchy<float>(c, c32);
}

paris_status solve_mixed(paris_ctx* c, const Coef<double>& c64, double* x, SolveOut& out,
                         int max_iter, bool rho0, bool half_rho) {
    const int64_t N = c->N;
    Level0Mode mode_guard{c};
    Coef<float> c32{c->b32_0[0], c->b32_0[1], c->b32_0[2], 1.0f};
    if (c->dirichlet) c32.sig = c->sig32_0;
    if (c->mixed_ready) {
        c->rho0 = rho0;
        c->half0 = !rho0 && c->opts.half_coefficients != 0 && !c->dirichlet;
    } else {
        mixed_setup(c, c64, rho0);
    }
    c->half_rho = c->rho0 && half_rho && c->rh16 && c->opts.level0_tiles == 1;
    c->lz = false;  // the same plane orders in every solve (the same sums)
    c->mixed_ready = false;
    // With the finest level from rho/2 the refinement step updates r in
    // double-float (launch_refine_rho) after the first FP64 residual; the
    // level-0 FP32 vectors are then in the colour-split layout, which only
    // the rho/2 kernels, the refinement step and the layout-free vector
    // kernels (dot products, axpy forms) touch.
    const bool refine = c->rho0;
    double prev_rr = INFINITY;
    int stalls = 0;
    for (bool first = true;; first = false) {
        // r32 = scale * (f - A x); x is the untouched initial guess on the first pass
        paris_status s = (first || !refine) ? true_residual(c, c64, x, c->r32, first, refine) : read_scal(c);
        if (first || !refine) c->lz = true;  // the residual ran through the planes in ascending order
        if (s != PARIS_OK) return s;
        const Scal& h = *c->scal_h;
        if (h.nonfinite > 0) { out.nonfinite = true; return PARIS_OK; }
        if (h.bnorm2 == 0.0 || meets(c, h)) { out.converged = true; return PARIS_OK; }
        if (out.iters >= max_iter) return PARIS_OK;
        if (h.rr > 0.25 * prev_rr) { if (++stalls >= 2) return PARIS_OK; } else stalls = 0;
        prev_rr = h.rr;
        ++out.outer;
        // inner solve of A e = r32 to a relative reduction inner_tol (not below
        // what the outer tolerance still needs, with a safety factor 0.1)
        const double rr32 = h.rr * h.scale * h.scale;
        double need2 = (c->opts.tol * c->opts.tol * h.bnorm2) / std::max(h.rr, 1e-300) * 1e-2;
        double it2 = c->opts.inner_tol * c->opts.inner_tol;
        const double target = rr32 * std::max(it2, std::min(need2, 1.0));
        // with the finest level from rho/2 the direction update d = z + beta d
        // rides in the next product (fuse_next: beta is pending), and so does
        // the previous iteration's update e += alpha d (e_pend), the last one
        // in the refinement step; e is written first by the second product
        // (e_mem), so it needs no clearing
        const bool fuse = c->rho0 && c->d32b && rho0_product_fuses(c->g0, c->opts.level0_tiles != 0);
        bool e_mem = !fuse, e_pend = false;
        if (!fuse) {
            ProfScope ps(c, PARIS_K_KRYLOV, 0.0);
            CK(cudaMemsetAsync(c->e32, 0, sizeof(float) * N, c->st));
        }
        vcycle<float>(c, c32, c->r32, c->z32);
        {
            ProfScope ps(c, PARIS_K_KRYLOV, 0.0);
            launch_dot2<float>(N, c->r32, c->z32, nullptr, c->partials, c->st,
                               FinSpec{c->scal, 2, 0, FIN_RHO_INIT, 0.0}, c->rho0 && take_dir(c));
            std::swap(c->d32, c->z32);  // first direction d = z: exchange the buffers
        }
        bool fuse_next = false;
        double prev_in_rr = rr32;  // ||r32||^2 before the last iteration
        for (int j = 0; j < 50 && out.iters < max_iter; ++j) {
            if (fuse_next) {
                // z, d, rho/2 and e (after the first) read; d, q and e written
                ProfScope ps(c, PARIS_K_MATVEC0, (5.0 + (e_pend ? (e_mem ? 3.0 : 2.0) : 0.0)) * N * 4);
                launch_matvec_rho_xpby(c->g0, c->rh32, c->grid.h, c->z32, c->d32, c->d32b, c->q32, c->scal,
                                       c->partials, c->st, FinSpec{c->scal, 1, 0, FIN_ALPHA, 0.0}, take_dir(c),
                                       e_pend ? c->e32 : nullptr, e_mem);
                if (e_pend) e_mem = true;
                e_pend = false;
                std::swap(c->d32, c->d32b);
            } else if (c->rho0) {
                ProfScope ps(c, PARIS_K_MATVEC0, 3.0 * N * 4);
                launch_matvec_rho(c->g0, c->rh32, c->grid.h, c->d32, c->q32, c->partials, c->st,
                                  FinSpec{c->scal, 1, 0, FIN_ALPHA, 0.0}, c->opts.level0_tiles != 0, take_dir(c));
            } else {
                ProfScope ps(c, PARIS_K_MATVEC0, (2.0 * N + beta_count(c->g0)) * 4);
                launch_matvec_dot<float>(c->g0, c32, c->d32, c->q32, c->partials, c->st,
                                         FinSpec{c->scal, 1, 0, FIN_ALPHA, 0.0});
            }
            {
                ProfScope ps(c, PARIS_K_KRYLOV, 0.0);
                if (fuse) {
                    launch_update_r<float>(N, c->scal, c->q32, c->r32, c->partials, c->st,
                                           FinSpec{c->scal, 3, 2, FIN_STORE, 0.0}, take_dir(c));
                    e_pend = true;  // e += alpha d, d = c->d32
                } else {
                    launch_update_xr<float>(N, c->scal, c->d32, c->q32, c->e32, c->r32, c->partials, c->st,
                                            FinSpec{c->scal, 3, 2, FIN_STORE, 0.0}, c->rho0 && take_dir(c));
                }
                s = read_scal_async(c);
                if (s != PARIS_OK) return s;
            }
            // the next iteration's V-cycle and dot products go in behind the
            // norms' copy while the host waits for it, when even a reduction
            // of ||r||^2 by 1000 in this iteration would leave it above the
            // target (the reduction per iteration is about 60 here); if the
            // iteration converges all the same, their results go unused
            const bool ahead = fuse && prev_in_rr * 1e-3 > target;
            auto next_direction = [&]() {
                vcycle<float>(c, c32, c->r32, c->z32);
                ProfScope ps(c, PARIS_K_KRYLOV, 0.0);
                launch_dot2<float>(N, c->z32, c->r32, c->q32, c->partials, c->st,  // (z.r, z.q)
                                   FinSpec{c->scal, 2, 0, FIN_FCG_BETA, 0.0}, c->rho0 && take_dir(c));
                if (fuse) {
                    fuse_next = true;
                } else {
                    launch_xpby<float>(N, c->scal, c->z32, c->d32, c->st);
                    c->lz = true;
                }
            };
            if (ahead) next_direction();
            {
                ProfScope ps(c, PARIS_K_KRYLOV, 0.0);
                s = read_scal_wait(c);
            }
            ++out.iters;
            if (s != PARIS_OK) return s;
            const double in_rr = c->scal_h->red[0];
            if (!(in_rr == in_rr) || c->scal_h->red[2] > 0) break;  // non-finite: the outer step decides
            if (in_rr <= target || in_rr > 1e6 * rr32) break;
            prev_in_rr = in_rr;
            if (!ahead) next_direction();
        }
        if (refine) {
            ProfScope ps(c, PARIS_K_RESID64, 48.0 * N);
            launch_refine_rho(c->g0, c->rh2, c->grid.h, c->e32, c->r, c->r, x, c->r32, c->scal, c->partials,
                              c->st, take_dir(c), e_mem, e_pend ? c->d32 : nullptr);
        } else {
            ProfScope ps(c, PARIS_K_KRYLOV, 0.0);
            launch_accumulate(N, c->scal, c->e32, x, c->st);
        }
        CK(cudaGetLastError());
    }
}

paris_status remove_mean(paris_ctx* c, double* x, int64_t n) {
    int64_t nb = launch_sum(n, x, c->partials, c->st);
    finalize(c->partials, nb, 3, 2, c->scal, FIN_STORE, 0.0, c->st);
    launch_sub_mean(n, x, c->scal, c->st);
    CK(cudaGetLastError());
    return PARIS_OK;
}

}  // namespace

// ================================================================== C ABI ===

extern "C" {

void paris_default_opts(paris_opts* o) {
    if (!o) return;
    o->tol = 1e-10;
    o->max_iter = 200;
    o->precision = PARIS_MIXED;
    o->nu1 = 2;
    o->nu2 = 2;
    o->omega = 1.15;
    o->smoother = PARIS_SMOOTH_RBGS_2PASS;
    o->coarse_max_cells = 8;
    o->inner_tol = 1e-5;
    o->fallback = 1;
    o->slab_planes = 0;
    o->half_coefficients = 0;
    o->level0_density = 1;
    o->level0_tiles = 1;
    o->level0_half_rho = 1;
    o->coarse_tail = 1;
}

const char* paris_status_string(paris_status s) {
    switch (s) {
        case PARIS_OK: return "ok";
        case PARIS_ERR_INVALID_ARG: return "invalid argument";
        case PARIS_ERR_CUDA: return "CUDA error";
        case PARIS_ERR_NOT_CONVERGED: return "not converged";
        case PARIS_ERR_NONFINITE: return "non-finite value";
        case PARIS_ERR_TIMEOUT: return "device wait timed out";
        case PARIS_ERR_NO_MEMORY: return "out of device memory";
    }
    return "unknown status";
}

paris_status paris_create(paris_ctx** out, const paris_grid* g, const paris_opts* o, void* stream) {
    if (!out) return PARIS_ERR_INVALID_ARG;
    *out = nullptr;
    paris_opts def;
    paris_default_opts(&def);
    if (!o) o = &def;
    if (!valid_grid(g) || !valid_opts(o)) return PARIS_ERR_INVALID_ARG;
    paris_ctx* c = new (std::nothrow) paris_ctx();
    if (!c) return PARIS_ERR_NO_MEMORY;
    c->grid = *g;
    c->opts = *o;
    c->g0 = Geo{g->nx, g->ny, g->nz, g->bc[0] == PARIS_WALL, g->bc[1] == PARIS_WALL,
                g->bc[2] == PARIS_WALL};
    c->N = c->g0.ncell();
    c->st = (cudaStream_t)stream;
    if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        c->cap_stream = nullptr;
    }
    paris_status s = alloc_ctx(c);
    if (s != PARIS_OK) {
        paris_destroy(c);
        return s;
    }
    *out = c;
    return PARIS_OK;
}

paris_status paris_destroy(paris_ctx* c) {
    if (!c) return PARIS_ERR_INVALID_ARG;
    cudaStreamSynchronize(c->st);
    drop_graphs(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->copy_st) {
        cudaStreamSynchronize(c->copy_st);
        cudaStreamDestroy(c->copy_st);
    }
    for (auto& e : c->copy_ev)
        if (e) cudaEventDestroy(e);
    if (c->scal_ev) cudaEventDestroy(c->scal_ev);
    c->mem.release();
    for (void* q : c->hw_mem) cudaFree(q);
    if (c->scal_h) cudaFreeHost(c->scal_h);
    for (auto& e : c->prof.ev) cudaEventDestroy(e);
    delete c;
    return PARIS_OK;
}

paris_status paris_set_opts(paris_ctx* c, const paris_opts* o) {
    if (!c || !valid_opts(o)) return PARIS_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(c->st));
    drop_graphs(c);  // sweeps and omega are baked into the captured V-cycle
    if (o->coarse_max_cells != c->opts.coarse_max_cells) {
        // the level plan depends on coarse_max_cells: rebuild the workspace
        CK(cudaStreamSynchronize(c->st));
        c->mem.release();
        if (c->scal_h) cudaFreeHost(c->scal_h);
        c->scal_h = nullptr;
        c->hC = c->hu = c->hv = c->hw = c->hp = nullptr;
        c->opts = *o;
        return alloc_ctx(c);
    }
    c->opts = *o;
    return PARIS_OK;
}

paris_status paris_profile(paris_ctx* c, int enable) {
    if (!c) return PARIS_ERR_INVALID_ARG;
    Profiler& P = c->prof;
    if (enable && P.ev.empty()) {
        P.ev.resize(2 * kProfPool);
        for (auto& e : P.ev) CK(cudaEventCreate(&e));
        P.slot_cls.resize(kProfPool);
        P.slot_bytes.resize(kProfPool);
        P.slot_n.resize(kProfPool);
    }
    if (enable) {
        CK(cudaStreamSynchronize(c->st));
        P.used = 0;
        for (int k = 0; k < PARIS_K_COUNT; ++k) P.launches[k] = 0;
    }
    P.on = enable != 0;
    return PARIS_OK;
}

paris_status paris_profile_read(paris_ctx* c, int cls, paris_kernel_prof* out) {
    if (!c || !out || cls < 0 || cls >= PARIS_K_COUNT) return PARIS_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(c->st));
    Profiler& P = c->prof;
    out->launches = P.launches[cls];
    out->timed = 0;
    out->ms = 0.0;
    out->bytes = 0.0;
    for (int s = 0; s < P.used; ++s) {
        if (P.slot_cls[s] != cls) continue;
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, P.ev[2 * s], P.ev[2 * s + 1]));
        out->timed += P.slot_n[s];
        out->ms += ms;
        out->bytes += P.slot_bytes[s];
    }
    return PARIS_OK;
}

int64_t paris_launch_count(void) { return (int64_t)launch_count(); }

const char* paris_last_cuda_error(void) { return last_cuda_error(); }

int64_t paris_face_count(const paris_ctx* c, int axis) {
    if (!c || axis < 0 || axis > 2) return -1;
    return c->g0.nface(axis);
}

int64_t paris_cell_count(const paris_ctx* c) { return c ? c->N : -1; }

paris_status paris_face_coeffs(paris_ctx* c, const double* C, double rho1, double rho2,
                               double* bx, double* by, double* bz) {
    if (!c || !C || !bx || !by || !bz) return PARIS_ERR_INVALID_ARG;
    if (!(rho1 > 0.0) || !(rho2 > 0.0) || !std::isfinite(rho1) || !std::isfinite(rho2))
        return PARIS_ERR_INVALID_ARG;
    launch_face_coeffs(c->g0, C, rho1, rho2, bx, by, bz, nullptr, nullptr, c->st);
    if (c->solid) launch_link_block(c->g0, c->solid, bx, by, bz, nullptr, nullptr, nullptr, c->st);
    CK(cudaGetLastError());
    return PARIS_OK;
}

paris_status paris_divergence(paris_ctx* c, const double* u, const double* v, const double* w,
                              double dt, double* rhs, double* mean_removed) {
    if (!c || !u || !v || !w || !rhs) return PARIS_ERR_INVALID_ARG;
    if (!(dt > 0.0) || !std::isfinite(dt)) return PARIS_ERR_INVALID_ARG;
    if (c->solid) {  // closed faces carry no flux; the mean over the fluid cells
        int64_t nb = launch_masked_divergence(c->g0, c->solid, u, v, w, 1.0 / (c->grid.h * dt), rhs, c->partials,
                                              c->st, no_fin());
        finalize(c->partials, nb, 3, 2, c->scal, FIN_MEAN_B, c->n_fluid, c->st);
        launch_fluid_sub_mean(c->N, c->solid, rhs, c->scal, c->st);
    } else {
        int64_t nb = launch_divergence(c->g0, u, v, w, 1.0 / (c->grid.h * dt), rhs, c->partials, c->st);
        finalize(c->partials, nb, 3, 2, c->scal, FIN_MEAN_B, (double)c->N, c->st);
        launch_sub_mean(c->N, rhs, c->scal, c->st);
    }
    CK(cudaGetLastError());
    if (mean_removed) {
        paris_status s = read_scal(c);
        if (s != PARIS_OK) return s;
        *mean_removed = c->scal_h->mean_b;
        c->last_mean_b = c->scal_h->mean_b;
    }
    return PARIS_OK;
}

}  // extern "C"

namespace {

// The solve behind paris_poisson_solve; rho0: the mixed form's level-0 FP32
// kernels rebuild their coefficients from rh32 (filled by the caller);
// mean_known: the caller reset scal and left the mean of rhs in scal->mean_b.
paris_status poisson_solve(paris_ctx* c, const double* bx, const double* by, const double* bz,
                           const double* rhs, double* p, paris_stats* st, bool rho0,
                           bool mean_known, bool half_rho = false) {
    const double ih2 = 1.0 / (c->grid.h * c->grid.h);
    Coef<double> c64{bx, by, bz, ih2};
    if (c->dirichlet) c64.sig = c->sig0;
    if (!mean_known) CK(cudaMemsetAsync(c->scal, 0, sizeof(Scal), c->st));
    paris_status s;
    {
        ProfScope ps(c, PARIS_K_SETUP, 0.0);
        s = prologue(c, rhs, p, mean_known);
    }
    if (s != PARIS_OK) return s;
    SolveOut out;
    int fell_back = 0;
    if (c->opts.precision == PARIS_MIXED && (!c->dirichlet || c->sig32_0)) {
        s = solve_mixed(c, c64, p, out, c->opts.max_iter, rho0, half_rho);
        if (s != PARIS_OK) return s;
        if (!out.converged && !out.nonfinite && c->opts.fallback) {
            SolveOut o2;
            s = solve_fp64(c, c64, p, o2, c->opts.max_iter, false);
            if (s != PARIS_OK) return s;
            o2.iters += out.iters;
            o2.outer += out.outer;
            out = o2;
            fell_back = 1;
        }
    } else {
        s = solve_fp64(c, c64, p, out, c->opts.max_iter, true);
        if (s != PARIS_OK) return s;
        out.outer = out.iters;
    }
    {
        ProfScope ps(c, PARIS_K_PROJECT, 0.0);
        if (c->dirichlet) {  // no null space: no gauge
            s = PARIS_OK;
        } else if (c->solid) {  // fluid mean 0, solid cells 0 (their p is not determined)
            launch_fluid_gauge(c->N, c->solid, p, c->partials, c->scal, c->st);
            CK(cudaGetLastError());
            s = PARIS_OK;
        } else {
            s = remove_mean(c, p, c->N);
        }
    }
    if (s != PARIS_OK) return s;
    s = read_scal(c);
    if (s != PARIS_OK) return s;
    const Scal& h = *c->scal_h;
    if (st) {
        st->iters = out.iters;
        st->outer_iters = out.outer;
        st->rel_res_l2 = h.bnorm2 > 0 ? std::sqrt(h.rr / h.bnorm2) : 0.0;
        st->rel_res_linf = h.binf > 0 ? h.rinf / h.binf : 0.0;
        st->mean_b_removed = h.mean_b;
        st->fell_back = fell_back;
        st->converged = out.converged ? 1 : 0;
        st->levels = (int)c->lv.size();
    }
    if (out.nonfinite) return PARIS_ERR_NONFINITE;
    return out.converged ? PARIS_OK : PARIS_ERR_NOT_CONVERGED;
}

}  // namespace

extern "C" {

paris_status paris_poisson_solve(paris_ctx* c, const double* bx, const double* by,
                                 const double* bz, const double* rhs, double* p,
                                 paris_stats* st) {
    if (!c || !bx || !by || !bz || !rhs || !p) return PARIS_ERR_INVALID_ARG;
    return poisson_solve(c, bx, by, bz, rhs, p, st, false, false);
}

paris_status paris_project(paris_ctx* c, const double* bx, const double* by, const double* bz,
                           const double* p, double dt, double* u, double* v, double* w) {
    if (!c || !bx || !by || !bz || !p || !u || !v || !w) return PARIS_ERR_INVALID_ARG;
    if (!(dt > 0.0) || !std::isfinite(dt)) return PARIS_ERR_INVALID_ARG;
    launch_project(c->g0, bx, by, bz, p, dt / c->grid.h, u, v, w, c->st);
    if (c->solid) launch_link_block(c->g0, c->solid, nullptr, nullptr, nullptr, u, v, w, c->st);  // blocked
    CK(cudaGetLastError());
    return PARIS_OK;
}

// Ordering against a copy stream for the host-buffer step: the compute
// stream waits for C before the face coefficients, for u*, v*, w* before the
// divergence and for p before the solve; p goes back to the host while the
// correction runs.
struct HostLink {
    cudaStream_t cs;
    cudaEvent_t c_ready, uvw_ready, p_ready, p_final;
    double* p_host;
};

paris_status projection_step_impl(paris_ctx* c, const double* C, double rho1, double rho2, double dt,
                                  double* u, double* v, double* w, double* p, paris_stats* st,
                                  const HostLink* hl, const Forcing* force = nullptr) {
    // the FP32 pairs of rho/2 need both half-densities well inside the FP32 range
    const double rlo = 0.5 * std::min(rho1, rho2), rhi = 0.5 * std::max(rho1, rho2);
    const bool use_rho0 = rho0_usable(c) && rlo >= 1e-30 && rhi <= 1e30;
    // FP16 rho/2 for the V-cycle (normal FP16 numbers with room to spare)
    const bool use_half = use_rho0 && !force && c->opts.level0_half_rho && c->rh16 && rlo >= 1e-4 && rhi <= 6e4 &&
                          rhi / rlo <= 1e7;
    c->rho_min = 2.0 * rlo;
    c->half_rho = use_half && c->opts.level0_tiles == 1;  // the set-up below writes level 1's FP16 copies
    // the set-up run ahead below is used by this step's solve only
    struct ReadyGuard {
        paris_ctx* c;
        ~ReadyGuard() { c->mixed_ready = false; }
    } ready_guard{c};
    {
        ProfScope ps(c, PARIS_K_FIELD, 0.0);
        if (hl) CK(cudaStreamWaitEvent(c->st, hl->c_ready, 0));
        if (use_rho0 && !force)  // beta to about 2^-46: the operator of the double-float refinement
            launch_face_coeffs_fast(c->g0, C, rho1, rho2, c->beta[0], c->beta[1], c->beta[2], c->rh32, c->rh2,
                                    use_half ? c->rh16 : nullptr, c->st);
        else
            launch_face_coeffs(c->g0, C, rho1, rho2, c->beta[0], c->beta[1], c->beta[2],
                               use_rho0 ? c->rh32 : nullptr, use_rho0 ? c->rh2 : nullptr, c->st, force);
        if (c->solid)
            launch_link_block(c->g0, c->solid, c->beta[0], c->beta[1], c->beta[2], nullptr, nullptr, nullptr, c->st);
        CK(cudaGetLastError());
    }
    if (c->opts.precision == PARIS_MIXED) {
        // the hierarchy needs the coefficients only: build it while the host
        // copies of u*, v*, w* and p may still be running
        const Coef<double> c64{c->beta[0], c->beta[1], c->beta[2], 1.0 / (c->grid.h * c->grid.h)};
        mixed_setup(c, c64, use_rho0);
        c->mixed_ready = true;
        CK(cudaGetLastError());
    }
    {
        ProfScope ps(c, PARIS_K_FIELD, 0.0);
        // rhs = div u*/dt and its mean; the solve's prologue forms the mean-free
        // f = -(rhs - mean) directly (no separate mean removal pass)
        CK(cudaMemsetAsync(c->scal, 0, sizeof(Scal), c->st));
        if (hl) CK(cudaStreamWaitEvent(c->st, hl->uvw_ready, 0));
        if (c->solid) {  // closed faces carry no flux; the mean over the fluid cells
            const int64_t nb = launch_masked_divergence(c->g0, c->solid, u, v, w, 1.0 / (c->grid.h * dt), c->rhs,
                                                        c->partials, c->st, no_fin());
            finalize(c->partials, nb, 3, 2, c->scal, FIN_MEAN_B, c->n_fluid, c->st);
        } else {
            const int64_t nb =
                launch_divergence(c->g0, u, v, w, 1.0 / (c->grid.h * dt), c->rhs, c->partials, c->st);
            finalize(c->partials, nb, 3, 2, c->scal, FIN_MEAN_B, (double)c->N, c->st);
        }
        CK(cudaGetLastError());
    }
    if (hl) CK(cudaStreamWaitEvent(c->st, hl->p_ready, 0));
    paris_status s;
    paris_status solve =
        poisson_solve(c, c->beta[0], c->beta[1], c->beta[2], c->rhs, p, st, use_rho0, true, use_half);
    if (solve != PARIS_OK && solve != PARIS_ERR_NOT_CONVERGED) return solve;
    if (hl) {
        // the correction only reads p: copy it out meanwhile
        CK(cudaEventRecord(hl->p_final, c->st));
        CK(cudaStreamWaitEvent(hl->cs, hl->p_final, 0));
        CK(cudaMemcpyAsync(hl->p_host, p, sizeof(double) * c->N, cudaMemcpyDeviceToHost, hl->cs));
    }
    {
        ProfScope ps(c, PARIS_K_PROJECT, 0.0);
        s = paris_project(c, c->beta[0], c->beta[1], c->beta[2], p, dt, u, v, w);
    }
    if (s != PARIS_OK) return s;
    return solve;
}

paris_status paris_projection_step(paris_ctx* c, const double* C, double rho1, double rho2,
                                   double dt, double* u, double* v, double* w, double* p,
                                   paris_stats* st) {
    if (!c || !C || !u || !v || !w || !p) return PARIS_ERR_INVALID_ARG;
    if (!(rho1 > 0.0) || !(rho2 > 0.0) || !std::isfinite(rho1) || !std::isfinite(rho2))
        return PARIS_ERR_INVALID_ARG;
    if (!(dt > 0.0) || !std::isfinite(dt)) return PARIS_ERR_INVALID_ARG;
    return projection_step_impl(c, C, rho1, rho2, dt, u, v, w, p, st, nullptr);
}

paris_status paris_set_solid(paris_ctx* c, const unsigned char* s) {
    if (!c) return PARIS_ERR_INVALID_ARG;
    if (!s) {
        c->solid = nullptr;
        c->n_fluid = 0.0;
        return PARIS_OK;
    }
    launch_fluid_count(c->N, s, c->partials, c->scal, c->st);
    CK(cudaGetLastError());
    paris_status st = read_scal(c);
    if (st != PARIS_OK) return st;
    const double n = c->scal_h->red[1];
    if (!(n >= 1.0)) return PARIS_ERR_INVALID_ARG;  // no fluid cell
    c->solid = s;
    c->n_fluid = n;
    return PARIS_OK;
}

paris_status paris_marker_function(paris_ctx* c, const double* gx, const double* gy, const double* gz,
                                   double mean_I, double* I, paris_stats* st) {
    if (!c || !gx || !gy || !gz || !I || !std::isfinite(mean_I)) return PARIS_ERR_INVALID_ARG;
    if (c->solid) return PARIS_ERR_INVALID_ARG;  // the marker is integrated on the whole grid
    // beta = 1 in the context's coefficient arrays, b = D G (h dt = h: dt = 1) and its mean
    launch_unit_beta(c->g0, c->beta[0], c->beta[1], c->beta[2], c->st);
    CK(cudaMemsetAsync(c->scal, 0, sizeof(Scal), c->st));
    const int64_t nb = launch_divergence(c->g0, gx, gy, gz, 1.0 / c->grid.h, c->rhs, c->partials, c->st);
    finalize(c->partials, nb, 3, 2, c->scal, FIN_MEAN_B, (double)c->N, c->st);
    CK(cudaGetLastError());
    const paris_status s = poisson_solve(c, c->beta[0], c->beta[1], c->beta[2], c->rhs, I, st, false, true);
    if (s != PARIS_OK && s != PARIS_ERR_NOT_CONVERGED) return s;
    launch_add_constant(c->N, I, mean_I, c->st);  // the solve left I mean-free
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->st));
    return s;
}

}  // extern "C"

namespace {

// The free-surface work arrays (all or nothing): the finest diagonal excess,
// one per coarse level, and two byte arrays of cell classes.
paris_status fs_alloc(paris_ctx* c) {
    if (c->sig0) return PARIS_OK;
    Alloc a;
    double* s0 = a.get<double>(c->N);
    float* s0f = a.get<float>(c->N);
    std::vector<double*> sl(c->lv.size(), nullptr);
    std::vector<float*> slf(c->lv.size(), nullptr);
    for (size_t l = 1; l < c->lv.size(); ++l) {
        sl[l] = a.get<double>(c->lv[l].g.ncell());
        slf[l] = a.get<float>(c->lv[l].g.ncell());
    }
    unsigned char* cls = a.get<unsigned char>(c->N);
    unsigned char* tmp = a.get<unsigned char>(c->N);
    if (a.err != cudaSuccess) {
        a.release();
        return PARIS_ERR_NO_MEMORY;
    }
    c->sig0 = s0;
    c->sig32_0 = s0f;
    for (size_t l = 1; l < c->lv.size(); ++l) {
        c->lv[l].sig64 = sl[l];
        c->lv[l].sig32 = slf[l];
    }
    c->fs_cls = cls;
    c->fs_tmp = tmp;
    c->mem.ptrs.insert(c->mem.ptrs.end(), a.ptrs.begin(), a.ptrs.end());
    return PARIS_OK;
}

// The projection on the unknown cells of c->fs_cls (1 unknown, 2 Dirichlet,
// 0 excluded): coefficients, diagonal excess and Dirichlet right-hand side,
// rhs = div u/dt - gd, the FP64 solve without null space, the cut-face
// velocity correction with coef = dt beta / h, the Dirichlet values into p.
paris_status fs_project_step(paris_ctx* c, const double* const theta[3], const double* pd, const double* kappa,
                             double sigma, double beta, double dt, bool zero_walls, double* u, double* v, double* w,
                             double* p, paris_stats* st) {
    launch_fs_setup(c->g0, c->fs_cls, beta, theta, pd, kappa, sigma, c->grid.h, c->beta[0], c->beta[1], c->beta[2],
                    c->sig0, c->rhs, c->st);
    launch_fs_rhs(c->g0, c->fs_cls, u, v, w, 1.0 / (c->grid.h * dt), c->rhs, c->st);
    CK(cudaMemsetAsync(c->scal, 0, sizeof(Scal), c->st));  // mean_b = 0: nothing is removed
    CK(cudaGetLastError());
    struct DirichletMode {
        paris_ctx* c;
        ~DirichletMode() { c->dirichlet = false; }
    } mode{c};
    c->dirichlet = true;
    c->mixed_ready = false;
    const paris_status solve = poisson_solve(c, c->beta[0], c->beta[1], c->beta[2], c->rhs, p, st, false, true);
    if (solve != PARIS_OK && solve != PARIS_ERR_NOT_CONVERGED) return solve;
    launch_fs_project(c->g0, c->fs_cls, theta, p, pd, kappa, sigma, dt * beta / c->grid.h, zero_walls, u, v, w,
                      c->st);
    launch_fs_fill(c->g0, c->fs_cls, pd, p, c->st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->st));
    return solve;
}

}  // namespace

extern "C" {

paris_status paris_free_surface_step(paris_ctx* c, const double* C, double rho_l, double dt, const double* theta_x,
                                     const double* theta_y, const double* theta_z, const double* kappa,
                                     double sigma, const double* p_gas, double* u, double* v, double* w, double* p,
                                     paris_stats* st) {
    if (!c || !C || !u || !v || !w || !p) return PARIS_ERR_INVALID_ARG;
    if (!(rho_l > 0.0) || !std::isfinite(rho_l) || !(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(sigma))
        return PARIS_ERR_INVALID_ARG;
    const bool any_t = theta_x || theta_y || theta_z, all_t = theta_x && theta_y && theta_z;
    if (any_t && !all_t) return PARIS_ERR_INVALID_ARG;
    if (c->solid) return PARIS_ERR_INVALID_ARG;
    paris_status s = fs_alloc(c);
    if (s != PARIS_OK) return s;
    launch_fs_liquid_classes(c->g0, C, c->fs_cls, c->st);
    const double* theta[3] = {theta_x, theta_y, theta_z};
    return fs_project_step(c, theta, p_gas, kappa, sigma, 1.0 / rho_l, dt, true, u, v, w, p, st);
}

paris_status paris_phantom_projection(paris_ctx* c, const double* C, double* u, double* v, double* w, double* phat,
                                      paris_stats* st) {
    if (!c || !C || !u || !v || !w || !phat) return PARIS_ERR_INVALID_ARG;
    if (c->solid) return PARIS_ERR_INVALID_ARG;
    paris_status s = fs_alloc(c);
    if (s != PARIS_OK) return s;
    launch_fs_gas_layers(c->g0, C, c->fs_tmp, c->fs_cls, c->st);
    const double* theta[3] = {nullptr, nullptr, nullptr};
    return fs_project_step(c, theta, nullptr, nullptr, 0.0, 1.0, 1.0, false, u, v, w, phat, st);
}

static bool valid_forcing(double sigma, double gx, double gy, double gz) {
    return std::isfinite(sigma) && sigma >= 0.0 && std::isfinite(gx) && std::isfinite(gy) && std::isfinite(gz);
}

paris_status paris_predictor_forcing(paris_ctx* c, const double* C, const double* kappa, double rho1,
                                     double rho2, double sigma, double gx, double gy, double gz, double tau,
                                     double* u, double* v, double* w, double* bx, double* by, double* bz) {
    if (!c || !C || !u || !v || !w || !bx || !by || !bz) return PARIS_ERR_INVALID_ARG;
    if (!(rho1 > 0.0) || !(rho2 > 0.0) || !std::isfinite(rho1) || !std::isfinite(rho2))
        return PARIS_ERR_INVALID_ARG;
    if (!valid_forcing(sigma, gx, gy, gz) || !std::isfinite(tau) || tau < 0.0) return PARIS_ERR_INVALID_ARG;
    const Forcing fo{kappa, sigma, c->grid.h, {gx, gy, gz}, tau, {u, v, w}};
    launch_face_coeffs(c->g0, C, rho1, rho2, bx, by, bz, nullptr, nullptr, c->st, &fo);
    CK(cudaGetLastError());
    return PARIS_OK;
}

paris_status paris_projection_step_forced(paris_ctx* c, const double* C, const double* kappa, double rho1,
                                          double rho2, double sigma, double gx, double gy, double gz,
                                          double dt, double* u, double* v, double* w, double* p,
                                          paris_stats* st) {
    if (!c || !C || !u || !v || !w || !p) return PARIS_ERR_INVALID_ARG;
    if (!(rho1 > 0.0) || !(rho2 > 0.0) || !std::isfinite(rho1) || !std::isfinite(rho2))
        return PARIS_ERR_INVALID_ARG;
    if (!(dt > 0.0) || !std::isfinite(dt) || !valid_forcing(sigma, gx, gy, gz)) return PARIS_ERR_INVALID_ARG;
    const Forcing fo{kappa, sigma, c->grid.h, {gx, gy, gz}, dt, {u, v, w}};
    return projection_step_impl(c, C, rho1, rho2, dt, u, v, w, p, st, nullptr, &fo);
}

paris_status paris_projection_step_host(paris_ctx* c, const double* C_host, double rho1,
                                        double rho2, double dt, double* u_host, double* v_host,
                                        double* w_host, double* p_host, paris_stats* st) {
    if (!c || !C_host || !u_host || !v_host || !w_host || !p_host) return PARIS_ERR_INVALID_ARG;
    const int64_t N = c->N;
    const int64_t nf[3] = {c->g0.nface(0), c->g0.nface(1), c->g0.nface(2)};
    if (!c->hC) {
        c->hC = c->mem.get<double>(N);
        c->hu = c->mem.get<double>(nf[0]);
        c->hv = c->mem.get<double>(nf[1]);
        c->hw = c->mem.get<double>(nf[2]);
        c->hp = c->mem.get<double>(N);
        if (c->mem.err != cudaSuccess) return PARIS_ERR_NO_MEMORY;
    }
    if (!(rho1 > 0.0) || !(rho2 > 0.0) || !std::isfinite(rho1) || !std::isfinite(rho2))
        return PARIS_ERR_INVALID_ARG;
    if (!(dt > 0.0) || !std::isfinite(dt)) return PARIS_ERR_INVALID_ARG;
    if (!c->copy_st) {
        // all or nothing: a failed creation leaves the context as it was
        cudaStream_t cs = nullptr;
        cudaEvent_t ev[5] = {};
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        for (int i = 0; i < 5 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (auto& x : ev)
                if (x) cudaEventDestroy(x);
            if (cs) cudaStreamDestroy(cs);
            paris_internal_note_cuda_error(e);
            return PARIS_ERR_CUDA;
        }
        c->copy_st = cs;
        for (int i = 0; i < 5; ++i) c->copy_ev[i] = ev[i];
    }
    cudaStream_t cs = c->copy_st;
    // on every way out, no copy into or out of the caller's buffers is left running
    struct DrainGuard {
        paris_ctx* c;
        ~DrainGuard() {
            cudaStreamSynchronize(c->copy_st);
            cudaStreamSynchronize(c->st);
        }
    } drain{c};
    // the copies start after the work already queued on the context's stream
    CK(cudaEventRecord(c->copy_ev[4], c->st));
    CK(cudaStreamWaitEvent(cs, c->copy_ev[4], 0));
    HostLink hl{cs, c->copy_ev[0], c->copy_ev[1], c->copy_ev[2], c->copy_ev[3], p_host};
    // inputs in the order the step needs them, each group announced by an event
    CK(cudaMemcpyAsync(c->hC, C_host, sizeof(double) * N, cudaMemcpyHostToDevice, cs));
    CK(cudaEventRecord(hl.c_ready, cs));
    CK(cudaMemcpyAsync(c->hu, u_host, sizeof(double) * nf[0], cudaMemcpyHostToDevice, cs));
    CK(cudaMemcpyAsync(c->hv, v_host, sizeof(double) * nf[1], cudaMemcpyHostToDevice, cs));
    CK(cudaMemcpyAsync(c->hw, w_host, sizeof(double) * nf[2], cudaMemcpyHostToDevice, cs));
    CK(cudaEventRecord(hl.uvw_ready, cs));
    CK(cudaMemcpyAsync(c->hp, p_host, sizeof(double) * N, cudaMemcpyHostToDevice, cs));
    CK(cudaEventRecord(hl.p_ready, cs));
    paris_status s = projection_step_impl(c, c->hC, rho1, rho2, dt, c->hu, c->hv, c->hw, c->hp, st, &hl);
    if (s != PARIS_OK && s != PARIS_ERR_NOT_CONVERGED) return s;
    // u, v, w go back once the correction is done (p is already on its way)
    CK(cudaEventRecord(c->copy_ev[4], c->st));
    CK(cudaStreamWaitEvent(cs, c->copy_ev[4], 0));
    CK(cudaMemcpyAsync(u_host, c->hu, sizeof(double) * nf[0], cudaMemcpyDeviceToHost, cs));
    CK(cudaMemcpyAsync(v_host, c->hv, sizeof(double) * nf[1], cudaMemcpyDeviceToHost, cs));
    CK(cudaMemcpyAsync(w_host, c->hw, sizeof(double) * nf[2], cudaMemcpyDeviceToHost, cs));
    CK(cudaStreamSynchronize(cs));
    CK(cudaStreamSynchronize(c->st));
    return s;
}

paris_status paris_project_adjoint(paris_ctx* c, const double* bx, const double* by,
                                   const double* bz, const double* p, double dt, const double* gu,
                                   const double* gv, const double* gw, double* gus, double* gvs,
                                   double* gws, double* gbx, double* gby, double* gbz, double* q,
                                   paris_stats* st) {
    if (!c || !bx || !by || !bz || !p || !gu || !gv || !gw || !gus || !gvs || !gws || !gbx || !gby ||
        !gbz || !q)
        return PARIS_ERR_INVALID_ARG;
    if (!(dt > 0.0) || !std::isfinite(dt)) return PARIS_ERR_INVALID_ARG;
    if (c->solid) return PARIS_ERR_INVALID_ARG;  // the adjoint of the blocking is not built
    const double inv_h = 1.0 / c->grid.h;
    // right-hand side of the adjoint solve: D (B g)
    launch_weighted_div(c->g0, bx, by, bz, gu, gv, gw, inv_h, c->rhs, c->partials, c->st);
    CK(cudaGetLastError());
    // the adjoint solve uses the same symmetric operator L = D B G
    paris_status solve = paris_poisson_solve(c, bx, by, bz, c->rhs, q, st);
    if (solve != PARIS_OK && solve != PARIS_ERR_NOT_CONVERGED) return solve;
    launch_adjoint_faces(c->g0, p, q, inv_h, dt, gu, gv, gw, gus, gvs, gws, gbx, gby, gbz, c->st);
    CK(cudaGetLastError());
    return solve;
}

paris_status paris_face_coeffs_adjoint(paris_ctx* c, double rho1, double rho2, const double* bx,
                                       const double* by, const double* bz, const double* gbx,
                                       const double* gby, const double* gbz, double* gC) {
    if (!c || !bx || !by || !bz || !gbx || !gby || !gbz || !gC) return PARIS_ERR_INVALID_ARG;
    if (!(rho1 > 0.0) || !(rho2 > 0.0) || !std::isfinite(rho1) || !std::isfinite(rho2))
        return PARIS_ERR_INVALID_ARG;
    launch_face_coeffs_adjoint(c->g0, rho1, rho2, bx, by, bz, gbx, gby, gbz, gC, c->st);
    CK(cudaGetLastError());
    return PARIS_OK;
}

paris_status paris_residual_norms(paris_ctx* c, const double* bx, const double* by,
                                  const double* bz, const double* rhs, const double* p,
                                  double* rel_l2, double* rel_linf) {
    if (!c || !bx || !by || !bz || !rhs || !p || !rel_l2 || !rel_linf) return PARIS_ERR_INVALID_ARG;
    const double ih2 = 1.0 / (c->grid.h * c->grid.h);
    Coef<double> c64{bx, by, bz, ih2};
    // f = -rhs as given (no mean removal): norms of rhs and of rhs - L p
    CK(cudaMemsetAsync(c->scal, 0, sizeof(Scal), c->st));
    int64_t nb = launch_make_rhs(c->N, rhs, c->scal, c->f, nullptr, c->partials, c->st);
    finalize(c->partials, nb, 4, 0xA, c->scal, FIN_BNORMS, 0.0, c->st);
    paris_status s = true_residual(c, c64, p, nullptr);
    if (s != PARIS_OK) return s;
    const Scal& h = *c->scal_h;
    *rel_l2 = h.bnorm2 > 0 ? std::sqrt(h.rr / h.bnorm2) : std::sqrt(h.rr);
    *rel_linf = h.binf > 0 ? h.rinf / h.binf : h.rinf;
    return PARIS_OK;
}

paris_status paris_check_arithmetic(const double* v, int64_t n, int shift, int64_t* mismatches,
                                    void* stream) {
    if (!v || !mismatches || n < 0 || shift > 60 || shift < -60) return PARIS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long* bad = nullptr;
    CK(cudaMalloc(&bad, sizeof(unsigned long long)));
    unsigned long long h = 0;
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess && n > 0) {
        launch_check_arithmetic(v, n, shift, bad, st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, bad, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(bad);
    if (e != cudaSuccess) {
        paris_internal_note_cuda_error(e);
        return PARIS_ERR_CUDA;
    }
    *mismatches = (int64_t)h;
    return PARIS_OK;
}

paris_status paris_stream_rates(const float* a, const float* b, const float* c, float* o, int64_t n, int reps,
                                double* read_gbs, double* triad_gbs, void* stream) {
    if (!a || !b || !c || !o || !read_gbs || !triad_gbs || n < 4 || n % 4 || reps < 1 || reps > 1000)
        return PARIS_ERR_INVALID_ARG;
    for (const void* p : {(const void*)a, (const void*)b, (const void*)c, (const void*)o})
        if (reinterpret_cast<uintptr_t>(p) & 15) return PARIS_ERR_INVALID_ARG;
    const cudaError_t e = stream_rates(a, b, c, o, n, reps, read_gbs, triad_gbs, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        paris_internal_note_cuda_error(e);
        return PARIS_ERR_CUDA;
    }
    return PARIS_OK;
}

paris_status paris_face_viscosity(paris_ctx* c, int comp, const double* C, double mu1, double mu2,
                                  double rho1, double rho2, double* nu) {
    if (!c || !C || !nu || comp < 0 || comp > 2) return PARIS_ERR_INVALID_ARG;
    if (!(mu1 > 0.0) || !(mu2 > 0.0) || !(rho1 > 0.0) || !(rho2 > 0.0) || !std::isfinite(mu1) ||
        !std::isfinite(mu2) || !std::isfinite(rho1) || !std::isfinite(rho2))
        return PARIS_ERR_INVALID_ARG;
    launch_helm_face_nu(helm_geo(c->g0, comp, c->grid.h), c->g0, C, mu1, mu2, rho1, rho2, nu, c->st);
    CK(cudaGetLastError());
    return PARIS_OK;
}

paris_status paris_viscous_solve(paris_ctx* c, int comp, const double* nu, double tau, const double* un,
                                 double* us, double tol, int max_iter, paris_stats* st) {
    if (!c || !nu || !un || !us || comp < 0 || comp > 2) return PARIS_ERR_INVALID_ARG;
    if (us == un || us == nu) return PARIS_ERR_INVALID_ARG;
    if (!(tau >= 0.0) || !std::isfinite(tau) || !(tol > 0.0 && tol < 1.0) || max_iter < 1)
        return PARIS_ERR_INVALID_ARG;
    if (st) *st = paris_stats{};
    const HelmGeo g = helm_geo(c->g0, comp, c->grid.h);
    CK(cudaMemsetAsync(c->scal, 0, sizeof(Scal), c->st));
    if (tau == 0.0) {  // u* = u^n
        launch_helm_init(g, un, nu, 1.0, us, c->partials, c->st, no_fin());
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(c->st));
        if (st) st->converged = 1;
        return PARIS_OK;
    }
    const auto met = [tol](const Scal& h) { return h.rr <= tol * tol * h.bnorm2 && h.rinf <= tol * h.binf; };
    const FinSpec rnorms{c->scal, 4, 2, FIN_RNORMS_RHO, 0.0};
    double *r = c->r, *z = c->z, *d = c->d, *q = c->q;
    launch_helm_init(g, un, nu, tau, us, c->partials, c->st, FinSpec{c->scal, 4, 0xA, FIN_BNORMS, 0.0});
    launch_helm_residual(g, un, nu, tau, us, r, z, c->partials, c->st, rnorms);
    CK(cudaGetLastError());
    paris_status s = read_scal(c);
    if (s != PARIS_OK) return s;
    int iters = 0, restarts = 0;
    bool converged = c->scal_h->bnorm2 == 0.0 || met(*c->scal_h);
    bool nonfinite = c->scal_h->nonfinite > 0;
    while (!converged && !nonfinite && iters < max_iter) {
        std::swap(d, z);  // first direction d = z: exchange the buffers
        bool inner = false;
        while (iters < max_iter) {
            launch_helm_matvec_dot(g, nu, tau, d, q, c->partials, c->st, FinSpec{c->scal, 1, 0, FIN_ALPHA, 0.0});
            launch_helm_update(g, nu, tau, c->scal, d, q, us, r, z, c->partials, c->st, rnorms);
            CK(cudaGetLastError());
            s = read_scal(c);
            if (s != PARIS_OK) return s;
            ++iters;
            if (c->scal_h->nonfinite > 0) { nonfinite = true; break; }
            if (met(*c->scal_h)) { inner = true; break; }
            launch_xpby<double>(helm_unknowns(g), c->scal, z, d, c->st);  // d = z + beta d
        }
        if (nonfinite) break;
        // verify with the true residual; restart from it if the recurrence drifted
        launch_helm_residual(g, un, nu, tau, us, r, z, c->partials, c->st, rnorms);
        CK(cudaGetLastError());
        s = read_scal(c);
        if (s != PARIS_OK) return s;
        nonfinite = c->scal_h->nonfinite > 0;
        converged = !nonfinite && met(*c->scal_h);
        if (converged || !inner || ++restarts > 3) break;
    }
    const Scal& h = *c->scal_h;
    if (st) {
        st->iters = iters;
        st->outer_iters = restarts + 1;
        st->rel_res_l2 = h.bnorm2 > 0 ? std::sqrt(h.rr / h.bnorm2) : 0.0;
        st->rel_res_linf = h.binf > 0 ? h.rinf / h.binf : 0.0;
        st->converged = converged ? 1 : 0;
    }
    if (nonfinite) return PARIS_ERR_NONFINITE;
    return converged ? PARIS_OK : PARIS_ERR_NOT_CONVERGED;
}

// The viscous multigrid's work arrays, allocated once per context: level l
// holds at most N / 8^l unknowns of any component (every axis is at least
// halved from one level to the next).
static paris_status helm_work(paris_ctx* c) {
    if (!c->hw_mem.empty()) return PARIS_OK;
    auto get = [&](size_t bytes, void** out) {
        if (cudaMalloc(out, bytes) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        c->hw_mem.push_back(*out);
        return true;
    };
    bool ok = get(sizeof(double) * (size_t)c->N, (void**)&c->hmg.sig64);
    int64_t n = c->N;
    for (int l = 0; ok && l < kHelmMaxLevels; ++l) {
        const size_t b = sizeof(float) * (size_t)std::max<int64_t>(n, 1);
        ok = get(b, (void**)&c->hmg.x[l]) && get(b, (void**)&c->hmg.f[l]) && get(b, (void**)&c->hmg.r[l]) &&
             get(b, (void**)&c->hmg.sig[l]);
        n = (n + 7) / 8;
    }
    if (!ok) {
        for (void* q : c->hw_mem) cudaFree(q);
        c->hw_mem.clear();
        c->hmg = HelmWork{};
        return PARIS_ERR_NO_MEMORY;
    }
    return PARIS_OK;
}

paris_status paris_viscous_solve_mg(paris_ctx* c, int comp, const double* nu, double tau, const double* un,
                                    double* us, double tol, int max_iter, paris_stats* st) {
    if (!c || !nu || !un || !us || comp < 0 || comp > 2) return PARIS_ERR_INVALID_ARG;
    if (us == un || us == nu) return PARIS_ERR_INVALID_ARG;
    if (!(tau >= 0.0) || !std::isfinite(tau) || !(tol > 0.0 && tol < 1.0) || max_iter < 1)
        return PARIS_ERR_INVALID_ARG;
    if (tau == 0.0) return paris_viscous_solve(c, comp, nu, tau, un, us, tol, max_iter, st);
    if (st) *st = paris_stats{};
    paris_status s = helm_work(c);
    if (s != PARIS_OK) return s;
    const HelmGeo g = helm_geo(c->g0, comp, c->grid.h);
    const HelmPlan P = helm_plan(g, kHelmMaxLevels);
    const int64_t n = helm_unknowns(g);
    const paris_opts& o = c->opts;
    const int nu1 = std::max(1, o.nu1), nu2 = std::max(1, o.nu2);
    const float omega = o.smoother == PARIS_SMOOTH_JACOBI ? 1.15f : (float)o.omega;
    CK(cudaMemsetAsync(c->scal, 0, sizeof(Scal), c->st));
    const auto met = [tol](const Scal& h) { return h.rr <= tol * tol * h.bnorm2 && h.rinf <= tol * h.binf; };
    const FinSpec rnorms{c->scal, 3, 2, FIN_RNORMS, 0.0};
    // FP64 iterative refinement around FP32 flexible CG: the FP64 residual of
    // the SPD form decides convergence; each refinement step solves A e = r
    // in FP32 with r scaled by a power of two (exact in both directions) to a
    // relative reduction inner_tol (or what the outer tolerance still needs)
    double* r = c->r;
    float *r32 = c->r32, *z32 = c->z32, *d32 = c->d32, *q32 = c->q32, *e32 = c->e32;
    launch_hmg_setup(g, un, nu, tau, c->hmg.sig64, c->hmg.sig[0], us, c->partials, c->st,
                     FinSpec{c->scal, 3, 2, FIN_BNORMS, 0.0});
    launch_hmg_sigma(P, c->hmg.sig, c->st);
    int iters = 0, outer = 0, stalls = 0;
    bool converged = false, nonfinite = false;
    double prev_rr = INFINITY;
    for (;;) {
        launch_hmg_residual64(g, un, c->hmg.sig64, us, r, c->partials, c->st, rnorms);
        CK(cudaGetLastError());
        s = read_scal(c);
        if (s != PARIS_OK) return s;
        const Scal& h = *c->scal_h;
        if (h.nonfinite > 0) { nonfinite = true; break; }
        if (h.bnorm2 == 0.0 || met(h)) { converged = true; break; }
        if (iters >= max_iter) break;
        if (h.rr > 0.25 * prev_rr) { if (++stalls >= 2) break; } else stalls = 0;
        prev_rr = h.rr;
        ++outer;
        finalize(c->partials, 0, 1, 0, c->scal, FIN_SCALE, 0.0, c->st);  // scale from max |r|
        launch_hmg_scale_d2f(n, r, c->scal, r32, c->partials, c->st, FinSpec{c->scal, 2, 2, FIN_STORE, 0.0});
        CK(cudaMemsetAsync(e32, 0, sizeof(float) * n, c->st));
        s = read_scal(c);
        if (s != PARIS_OK) return s;
        const double rr32 = c->scal_h->red[0];
        const double need2 = (tol * tol * h.bnorm2) / std::max(h.rr, 1e-300) * 1e-2;
        const double it2 = o.inner_tol * o.inner_tol;
        const double target = rr32 * std::max(it2, std::min(need2, 1.0));
        launch_hmg_vcycle32(P, c->hmg, r32, z32, nu1, nu2, 8, omega, c->st);
        launch_dot2<float>(n, r32, z32, nullptr, c->partials, c->st, FinSpec{c->scal, 2, 0, FIN_RHO_INIT, 0.0});
        std::swap(d32, z32);  // first direction d = z
        for (int j = 0; j < 50 && iters < max_iter; ++j) {
            launch_hmg_matvec32(P, c->hmg.sig[0], d32, q32, c->partials, c->st, FinSpec{c->scal, 1, 0, FIN_ALPHA, 0.0});
            launch_update_xr<float>(n, c->scal, d32, q32, e32, r32, c->partials, c->st,
                                    FinSpec{c->scal, 3, 2, FIN_STORE, 0.0});
            CK(cudaGetLastError());
            s = read_scal(c);
            if (s != PARIS_OK) return s;
            ++iters;
            const double in_rr = c->scal_h->red[0];
            if (!(in_rr == in_rr) || c->scal_h->red[2] > 0) break;  // non-finite: the FP64 residual decides
            if (in_rr <= target || in_rr > 1e6 * rr32) break;
            launch_hmg_vcycle32(P, c->hmg, r32, z32, nu1, nu2, 8, omega, c->st);
            // flexible CG(1): beta = -(z . q) / (d . q) with the new z
            launch_dot2<float>(n, z32, r32, q32, c->partials, c->st, FinSpec{c->scal, 2, 0, FIN_FCG_BETA, 0.0});
            launch_xpby<float>(n, c->scal, z32, d32, c->st);
        }
        launch_hmg_accumulate(g, e32, c->scal, us, c->st);  // u* += e / scale
        CK(cudaGetLastError());
    }
    const Scal& h = *c->scal_h;
    if (st) {
        st->iters = iters;
        st->outer_iters = outer;
        st->rel_res_l2 = h.bnorm2 > 0 ? std::sqrt(h.rr / h.bnorm2) : 0.0;
        st->rel_res_linf = h.binf > 0 ? h.rinf / h.binf : 0.0;
        st->converged = converged ? 1 : 0;
        st->levels = P.nl;
    }
    if (nonfinite) return PARIS_ERR_NONFINITE;
    return converged ? PARIS_OK : PARIS_ERR_NOT_CONVERGED;
}

paris_status paris_max_divergence(paris_ctx* c, const double* u, const double* v,
                                  const double* w, double* max_abs_div) {
    if (!c || !u || !v || !w || !max_abs_div) return PARIS_ERR_INVALID_ARG;
    int64_t nb = launch_max_divergence(c->g0, u, v, w, 1.0 / c->grid.h, c->partials, c->st);
    finalize(c->partials, nb, 1, 1, c->scal, FIN_STORE, 0.0, c->st);
    CK(cudaGetLastError());
    paris_status s = read_scal(c);
    if (s != PARIS_OK) return s;
    *max_abs_div = c->scal_h->red[0];
    return PARIS_OK;
}

}  // extern "C"
