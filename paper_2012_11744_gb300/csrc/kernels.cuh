// Host-side launchers of the projection kernels (internal to the library).
#pragma once

#include <utility>

#include "common.cuh"

namespace paris {

// Device-resident scalars of one solve; written by finalize_kernel, read by
// the kernels that need them (no host round trip inside an iteration).
struct Scal {
    double red[4];       // last finalized reduction results
    double mean_b;       // mean removed from the right-hand side
    double bnorm2;       // ||f||_2^2 of the mean-free right-hand side
    double binf;         // ||f||_inf
    double rho;          // (F)CG: r . z
    double alpha;        // (F)CG step length
    double beta;         // (F)CG direction update coefficient
    double rr;           // current residual ||r||_2^2
    double rinf;         // current residual ||r||_inf
    double scale;        // MIXED: r32 = scale * r64; correction e64 = e32 / scale (a power of 2)
    double inv_scale;
    double scale_exp;    // log2(scale), an integer
    double rr0;          // MIXED: ||r32||_2^2 at the start of the inner solve
    double nonfinite;    // > 0 if a NaN/Inf was seen
    double xmax;         // max |x| of the initial guess (0: the first residual is f)
    unsigned ticket;     // blocks of the running reduction that stored their partials
    unsigned wait_fail;  // a bounded device-side wait gave up (staged kernels)
};

enum FinalizeMode {
    FIN_STORE = 0,      // red[q] = result q
    FIN_MEAN_B = 1,     // mean_b = result0 / param
    FIN_BNORMS = 2,     // bnorm2 = result0, binf = result1
    FIN_RNORMS = 3,     // rr = result0, rinf = result1
    FIN_ALPHA = 4,      // alpha = rho / result0
    FIN_RHO_BETA = 5,   // beta = result0 / rho, rho = result0 (PCG)
    FIN_RHO_INIT = 6,   // rho = result0 (first direction)
    FIN_FCG_BETA = 7,   // beta = -alpha * result1 / rho, rho = result0 (flexible CG)
    FIN_SCALE = 8,      // scale = 1/max(result1, tiny), rr0 = rr*scale^2 ... (mixed)
    FIN_INNER_INIT = 9, // rr0 = result0, rr = result0
    FIN_REFINE = 10,    // scale from the current rinf, then rr = result0 / scale^2, rinf = result1
    FIN_RNORMS_RHO = 11, // rr = result0, rinf = result1, beta = result3 / rho, rho = result3 (Jacobi PCG)
    FIN_MEAN_FLUID = 12  // mean_b = result0 / result1 (a sum and a count over the fluid cells)
};

// Second stage of a reduction, by one block of kRedThreads threads: fold the
// nv values of nblocks block partials in a fixed order (four interleaved
// accumulators per thread, then the warps, then the block), store them in
// s->red and apply `mode`.  Deterministic: the order depends only on nblocks.
__device__ inline void finalize_block(const double* partials, int64_t nblocks, int nv, int maxmask, Scal* s,
                                      int mode, double param, int tid) {
    __shared__ double sh[kRedThreads / 32][4];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int q = 0; q < nv; ++q) {
        const bool mx = (maxmask >> q) & 1;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int64_t b = tid;
        // partials written by other blocks of this launch: read past L1
        for (; b + 3 * kRedThreads < nblocks; b += 4 * kRedThreads) {
            const double t0 = __ldcg(partials + (int64_t)nv * b + q);
            const double t1 = __ldcg(partials + (int64_t)nv * (b + kRedThreads) + q);
            const double t2 = __ldcg(partials + (int64_t)nv * (b + 2 * kRedThreads) + q);
            const double t3 = __ldcg(partials + (int64_t)nv * (b + 3 * kRedThreads) + q);
            if (mx) { a0 = fmax(a0, t0); a1 = fmax(a1, t1); a2 = fmax(a2, t2); a3 = fmax(a3, t3); }
            else { a0 += t0; a1 += t1; a2 += t2; a3 += t3; }
        }
        for (; b < nblocks; b += kRedThreads) {
            const double t0 = __ldcg(partials + (int64_t)nv * b + q);
            a0 = mx ? fmax(a0, t0) : a0 + t0;
        }
        v[q] = mx ? fmax(fmax(a0, a1), fmax(a2, a3)) : (a0 + a1) + (a2 + a3);
    }
    const int lane = tid & 31, wid = tid >> 5;
    for (int q = 0; q < 4; ++q) {
        v[q] = ((maxmask >> q) & 1) ? warp_max(v[q]) : warp_sum(v[q]);
        if (lane == 0) sh[wid][q] = v[q];
    }
    __syncthreads();
    if (tid == 0) {
        double r[4];
        for (int q = 0; q < 4; ++q) {
            double t = 0.0;
            for (int w = 0; w < kRedThreads / 32; ++w)
                t = ((maxmask >> q) & 1) ? fmax(t, sh[w][q]) : t + sh[w][q];
            r[q] = t;
            s->red[q] = t;
        }
        // r32 = scale * r64 keeps the FP32 inner problem O(1): scale is the
        // power of two that maps max |r| into [0.5, 1), so scaling is an exact
        // exponent shift in both directions (taken from the previous residual,
        // kept until its FP32 correction has been accumulated)
        auto set_scale = [&]() {
            const double m = s->rinf > 1e-300 && isfinite(s->rinf) ? s->rinf : 1.0;
            int ex = 0;
            frexp(m, &ex);
            s->scale = ldexp(1.0, -ex);
            s->inv_scale = ldexp(1.0, ex);
            s->scale_exp = (double)(-ex);
        };
        switch (mode) {
            case FIN_MEAN_B: s->mean_b = r[0] / param; s->nonfinite += r[2]; break;
            case FIN_BNORMS:  // the first residual of a solve is f itself: seed rinf with |f|inf
                s->bnorm2 = r[0]; s->binf = r[1]; s->rinf = r[1]; s->nonfinite += r[2];
                s->xmax = r[3];
                break;
            case FIN_RNORMS: s->rr = r[0]; s->rinf = r[1]; s->nonfinite += r[2]; break;
            case FIN_RNORMS_RHO:
                s->rr = r[0]; s->rinf = r[1]; s->nonfinite += r[2];
                s->beta = (s->rho != 0.0) ? r[3] / s->rho : 0.0;
                s->rho = r[3];
                break;
            case FIN_ALPHA: s->alpha = (r[0] > 0.0) ? s->rho / r[0] : 0.0; break;
            case FIN_RHO_BETA: s->beta = (s->rho != 0.0) ? r[0] / s->rho : 0.0; s->rho = r[0]; break;
            case FIN_RHO_INIT: s->rho = r[0]; s->beta = 0.0; break;
            case FIN_MEAN_FLUID: s->mean_b = r[1] > 0.0 ? r[0] / r[1] : 0.0; break;
            case FIN_FCG_BETA:
                s->beta = (s->rho != 0.0) ? -s->alpha * r[1] / s->rho : 0.0;
                s->rho = r[0];
                break;
            case FIN_SCALE: set_scale(); break;
            case FIN_INNER_INIT: s->rr0 = r[0]; s->rr = r[0]; s->rinf = r[1]; break;
            case FIN_REFINE:  // the refinement step scaled its r32 by max |r| before the
                              // step and summed the squares of r32
                set_scale();
                s->rr = r[0] * s->inv_scale * s->inv_scale;
                s->rinf = r[1];
                s->nonfinite += r[2];
                break;
            default: break;
        }
    }
}

// A reduction's second stage fused into its first: `s` null means none (the
// caller launches finalize).  Otherwise every block, after storing its
// partials (thread 0 writes them), takes a ticket; the block that takes the
// last one folds all partials (finalize_block) and resets the ticket.
struct FinSpec {
    Scal* s;
    int nv, maxmask, mode;
    double param;
};
inline FinSpec no_fin() { return FinSpec{nullptr, 0, 0, 0, 0.0}; }

__device__ inline void finalize_last_block(const double* partials, int64_t nblocks, const FinSpec& f, int tid) {
    if (!f.s) return;
    __shared__ bool last;
    if (tid == 0) {
        __threadfence();  // this block's partials before its ticket
        const unsigned t = atomicAdd(&f.s->ticket, 1u);
        last = t == (unsigned)(nblocks - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();  // every other block's partials before the fold
    finalize_block(partials, nblocks, f.nv, f.maxmask, f.s, f.mode, f.param, tid);
    if (tid == 0) f.s->ticket = 0u;
}

// Best-of-reps device rates of two streams over n-float vectors (n a
// multiple of 4, 16-byte aligned): a, b, c read (read_gbs) and o = a + b/2
// (triad_gbs, two read and one written), bytes moved over event time.
cudaError_t stream_rates(const float* a, const float* b, const float* c, float* o, int64_t n, int reps,
                         double* read_gbs, double* triad_gbs, cudaStream_t st);

// Launch with programmatic stream serialization: the launch is processed
// while the preceding kernel on the stream runs, and the kernel (which must
// call pdl_wait() before reading that kernel's results) starts as soon as
// the preceding kernel completes.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Streaming multiprocessors of the current device (queried once per device).
int device_sms();
// Grid of the element-wise kernels (kEW elements per thread).
int elementwise_blocks(int64_t n);
// Most blocks any reducing kernel launches on a grid of this size (the
// number of partial-sum slots a caller must provide, per value).
int64_t max_reduce_blocks(const Geo& g);

// Remember the last CUDA error seen by the library (for paris_last_cuda_error).
void paris_internal_note_cuda_error(cudaError_t e);
const char* last_cuda_error();

// Process-wide count of kernel launches made by the library.
void count_launch(int n = 1);
long long launch_count();

void finalize(const double* partials, int64_t nblocks, int nv, int maxmask, Scal* s, int mode,
              double param, cudaStream_t st);

// ------------------------------------------------------------ solid cells ---
// Sec. 3.8 "Lego" solids (solid.cu): s = 1 outside the solid, 0 inside; a
// face is open when both of its cells are fluid.
// beta and/or u zeroed on every closed face (pointers may be null)
void launch_link_block(const Geo& g, const unsigned char* s, double* bx, double* by, double* bz, double* u,
                       double* v, double* w, cudaStream_t st);
// rhs = div u/(h dt) with closed faces carrying no flux, 0 in solid cells;
// partials (sum, max |rhs|, non-finite count) on the divergence's grid
int64_t launch_masked_divergence(const Geo& g, const unsigned char* s, const double* u, const double* v,
                                 const double* w, double inv_hdt, double* rhs, double* partials, cudaStream_t st,
                                 FinSpec fin);
// x <- x - (mean over the fluid cells), 0 in solid cells (the gauge)
void launch_fluid_gauge(int64_t n, const unsigned char* s, double* x, double* partials, Scal* sc, cudaStream_t st);
// x <- x - sc->mean_b on fluid cells, 0 in solid cells
void launch_fluid_sub_mean(int64_t n, const unsigned char* s, double* x, const Scal* sc, cudaStream_t st);
// sc->mean_b = mean of x over the fluid cells
void launch_fluid_mean(int64_t n, const unsigned char* s, const double* x, double* partials, Scal* sc,
                       cudaStream_t st);
// x <- 0 in solid cells
void launch_solid_zero(int64_t n, const unsigned char* s, double* x, cudaStream_t st);
// sc->red[1] = number of fluid cells; returns the blocks used
int64_t launch_fluid_count(int64_t n, const unsigned char* s, double* partials, Scal* sc, cudaStream_t st);

// marker function (Eq. FrontMarker3): beta = 1 on every face, 0 on walls;
// x += a on n entries
void launch_unit_beta(const Geo& g, double* bx, double* by, double* bz, cudaStream_t st);
void launch_add_constant(int64_t n, double* x, double a, cudaStream_t st);

// free-surface projections (Sec. 3.7.5, freesurf.cu).  Cell classes: 1
// unknown, 2 Dirichlet, 0 excluded.
// liquid (C < 1/2) unknown, gas Dirichlet
void launch_fs_liquid_classes(const Geo& g, const double* C, unsigned char* cls, cudaStream_t st);
// the first two gas layers unknown, the liquid excluded, the gas beyond Dirichlet (tmp: scratch)
void launch_fs_gas_layers(const Geo& g, const double* C, unsigned char* tmp, unsigned char* cls, cudaStream_t st);
// beta on the faces between unknown cells (0 elsewhere), the diagonal excess
// sig (sum of beta/theta over the Dirichlet faces) and gd = sum of
// beta/(theta h^2) p_s, p_s = pd[d] + sigma (kappa_c + kappa_d)/2 (null pd,
// kappa, theta: 0, 0, 1)
void launch_fs_setup(const Geo& g, const unsigned char* cls, double beta, const double* const theta[3],
                     const double* pd, const double* kappa, double sigma, double h, double* bx, double* by,
                     double* bz, double* sig, double* gd, cudaStream_t st);
// rhs = div u/(h dt) - gd on the unknown cells, 0 elsewhere (gd read from rhs)
void launch_fs_rhs(const Geo& g, const unsigned char* cls, const double* u, const double* v, const double* w,
                   double inv_hdt, double* rhs, cudaStream_t st);
// u -= coef (cut-face gradient) on the faces touching an unknown cell
void launch_fs_project(const Geo& g, const unsigned char* cls, const double* const theta[3], const double* p,
                       const double* pd, const double* kappa, double sigma, double coef, bool zero_walls,
                       double* u, double* v, double* w, cudaStream_t st);
// p = pd (Dirichlet cells; 0 without pd) or 0 (excluded cells)
void launch_fs_fill(const Geo& g, const unsigned char* cls, const double* pd, double* p, cudaStream_t st);

// ------------------------------------------------- implicit viscous step ---
// One velocity component of Sec. 3.2.3 (Eq. muelliptic) in SPD form,
// (diag(1/(tau nu)) - Lap_h) u* = u^n/(tau nu), on its unknowns (viscous.cu).

enum HelmKind { HELM_PERIODIC = 0, HELM_ZERO = 1, HELM_NOSLIP = 2 };

struct HelmGeo {
    int m[3];     // unknowns along x, y, z
    int e[3];     // extents of the component's full face array
    int kind[3];  // beyond the ends of each axis: wrap, zero, minus the end value
    int comp;     // 0 = u (x-faces), 1 = v, 2 = w
    int wall;     // the face array holds wall faces along the component's axis
    int64_t off;  // face-array index of unknown (0,0,0)
    double ih2;   // 1/h^2
};
HelmGeo helm_geo(const Geo& g0, int comp, double h);

// Multigrid preconditioner of the viscous step (helmmg.cu): per level the
// unknowns per axis, the axis kinds and 1/h_l^2; the FP32 work arrays.
constexpr int kHelmMaxLevels = 10;
struct HelmLevelDesc {
    int m[3];
    int kind[3];
    double ih2;
};
struct HelmPlan {
    int nl;
    HelmLevelDesc lv[kHelmMaxLevels];
};
struct HelmWork {
    float* x[kHelmMaxLevels];
    float* f[kHelmMaxLevels];
    float* r[kHelmMaxLevels];
    float* sig[kHelmMaxLevels];
    double* sig64;
};
// coarsen every axis together while each can (periodic / no-slip: even and
// >= 4; the component's own wall axis: odd and >= 5)
HelmPlan helm_plan(const HelmGeo& g, int max_levels);
// sigma = 1/(tau nu) (FP64 and level-0 FP32), u* = u^n on the unknowns and 0
// on the own wall faces; partials of |b|^2, max |b|, non-finite (b = sigma u^n)
int64_t launch_hmg_setup(const HelmGeo& g, const double* un, const double* nu, double tau, double* sig64,
                         float* sig32, double* us, double* partials, cudaStream_t st, FinSpec fin);
// the coarse levels' sigma by restriction
void launch_hmg_sigma(const HelmPlan& P, float* const* sig, cudaStream_t st);
// r = sigma u^n - A u*; partials (|r|^2, max |r|, non-finite)
int64_t launch_hmg_residual64(const HelmGeo& g, const double* un, const double* sig, const double* us, double* r,
                              double* partials, cudaStream_t st, FinSpec fin);
int64_t helm_max_blocks(const HelmGeo& g);
// FP32 inner iteration of the mixed form: z32 = V r32 (finest-level vectors
// given, not the work arrays); q = A d in FP32 and d . q; r32 = scale r64 and
// its norms (scale from the scalar block); u* += e / scale
void launch_hmg_vcycle32(const HelmPlan& P, const HelmWork& W, const float* r32, float* z32, int nu1, int nu2,
                         int coarse_sweeps, float omega, cudaStream_t st);
int64_t launch_hmg_matvec32(const HelmPlan& P, const float* sig, const float* d, float* q, double* partials,
                            cudaStream_t st, FinSpec fin);
int64_t launch_hmg_scale_d2f(int64_t n, const double* r, const Scal* s, float* r32, double* partials,
                             cudaStream_t st, FinSpec fin);
void launch_hmg_accumulate(const HelmGeo& g, const float* e, const Scal* s, double* us, cudaStream_t st);
int64_t helm_unknowns(const HelmGeo& g);
int64_t helm_faces(const HelmGeo& g);
// us = un on the unknowns, 0 on the wall faces; partials (|b|^2, max|b|,
// non-finite count, 0) of b = un/(tau nu)
int64_t launch_helm_init(const HelmGeo& g, const double* un, const double* nu, double tau, double* us,
                         double* partials, cudaStream_t st, FinSpec fin);
// r = b - A x, z = r/diag(A); partials (r.r, max|r|, non-finite count, r.z)
int64_t launch_helm_residual(const HelmGeo& g, const double* un, const double* nu, double tau, const double* x,
                             double* r, double* z, double* partials, cudaStream_t st, FinSpec fin);
// q = A d; partials d.q
int64_t launch_helm_matvec_dot(const HelmGeo& g, const double* nu, double tau, const double* d, double* q,
                               double* partials, cudaStream_t st, FinSpec fin);
// x += alpha d, r -= alpha q, z = r/diag(A); partials as launch_helm_residual
int64_t launch_helm_update(const HelmGeo& g, const double* nu, double tau, const Scal* s, const double* d,
                           const double* q, double* x, double* r, double* z, double* partials, cudaStream_t st,
                           FinSpec fin);
// nu_f = (mu_L + mu_R)/(rho_L + rho_R) on the component's faces, 0 on its wall faces
void launch_helm_face_nu(const HelmGeo& g, const Geo& g0, const double* C, double mu1, double mu2, double rho1,
                         double rho2, double* nu, cudaStream_t st);

// ---------------------------------------------------------- field steps ---
// beta = 2/(rho_L + rho_R) (FP64); rh32 (may be null): FP32 copy of rho/2,
// rh2 (may be null): rho/2 as (hi, lo) FP32 pairs, hi = rh32
// The predictor's capillary and gravity forcing fused into the face
// coefficients (Eqs. nonconspredictedvel, csf2): u* = u^n + tau a_f in place.
struct Forcing {
    const double* kappa;  // cell curvature (null: 0)
    double sigma, h;      // surface tension, cell size
    double g[3];          // gravity per axis
    double tau;           // predictor time step
    double* u[3];         // face arrays: in u^n, out u*
};
void launch_face_coeffs(const Geo& g, const double* C, double rho1, double rho2, double* bx,
                        double* by, double* bz, float* rh32, float2* rh2, cudaStream_t st,
                        const Forcing* force = nullptr);
// the same outputs (rh32, rh2 required) with beta from the rho/2 pairs in FP32
// arithmetic: within about 2^-46 of 1/rho_f (the mixed form's step); rh16 (may
// be null): rho/2 in FP16 (rounded from rh32)
void launch_face_coeffs_fast(const Geo& g, const double* C, double rho1, double rho2, double* bx, double* by,
                             double* bz, float* rh32, float2* rh2, __half* rh16, cudaStream_t st);
// rhs = div(u)/(h dt); partials: (sum rhs, max |rhs|, nonfinite count)
int64_t launch_divergence(const Geo& g, const double* u, const double* v, const double* w,
                          double inv_hdt, double* rhs, double* partials, cudaStream_t st,
                          FinSpec fin = no_fin());
// f = -(rhs - mean_b), partials: (||f||^2, max|f|, nonfinite, max|x0|); x0 (the
// initial guess) may be null
int64_t launch_make_rhs(int64_t n, const double* rhs, const Scal* s, double* f, const double* x0,
                        double* partials, cudaStream_t st, FinSpec fin = no_fin(), const unsigned char* solid = nullptr);
void launch_sub_mean(int64_t n, double* x, const Scal* s, cudaStream_t st);
int64_t launch_sum(int64_t n, const double* x, double* partials, cudaStream_t st);
void launch_project(const Geo& g, const double* bx, const double* by, const double* bz,
                    const double* p, double dt_over_h, double* u, double* v, double* w,
                    cudaStream_t st);
int64_t launch_max_divergence(const Geo& g, const double* u, const double* v, const double* w,
                              double inv_h, double* partials, cudaStream_t st);

// ---------------------------------------------------- level set-up --------
template <typename T>
void launch_convert_beta(const Geo& g, const double* b64[3], double scale, T* out[3],
                         cudaStream_t st);
// out = float(in * scale) over n cells (the FP32 copy of a diagonal excess)
void launch_convert_scaled(int64_t n, const double* in, double scale, float* out, cudaStream_t st);
template <typename T>
void launch_coarse_beta(const Geo& fine, const Coef<T>& cf, const Geo& coarse, const int f[3],
                        const double hc2_over_hf2[3], T* out[3], cudaStream_t st);
template <typename T>
void launch_inv_diag(const Geo& g, const Coef<T>& cf, T* w, cudaStream_t st);
// dense (A + a 1 1^T)^{-1} of the coarsest operator, FP64, one CTA
template <typename T>
void launch_coarse_inverse(const Geo& g, const Coef<T>& cf, double* inv, cudaStream_t st);
// x = inv (f - mean f); keep_mean: x = inv f (an operator without null space)
template <typename T>
void launch_coarse_solve(const Geo& g, const double* inv, const T* f, T* x, cudaStream_t st, bool keep_mean);
// coarse diagonal excess (Coef::sig) from the fine one of a level with the given scale
template <typename T>
void launch_coarse_sig(const Geo& fine, const T* sig, double scale, const Geo& coarse, const int f[3], T* out,
                       cudaStream_t st);

// ------------------------------------------------------------ V-cycle -----
// One red-black colour pass of over-relaxed Gauss-Seidel on A x = f, in
// place, on the z-planes [k0, k1) (k1 < 0: all planes).
// zero_init: x is taken as 0 on entry (the pass also zeroes the other colour).
template <typename T>
void launch_rbgs(const Geo& g, const Coef<T>& cf, const T* w, const T* f, T* x, int color,
                 double omega, bool zero_init, cudaStream_t st, int k0 = 0, int k1 = -1);
// One fused red-black sweep (both colours, one pass) from xin to xout
// (separate arrays; xin unread when zero_init).  first_color: colour
// updated first (0 = red, (i+j+k) even).  use_w: read the inverse diagonal
// from w instead of recomputing it from the coefficients.
template <typename T>
void launch_rbgs_fused(const Geo& g, const Coef<T>& cf, const T* w, const T* f, const T* xin,
                       T* xout, int first_color, double omega, bool zero_init, bool use_w,
                       cudaStream_t st);
// The fused sweep indexes with 32-bit integers: true when the level fits.
bool rbgs_fused_fits(const Geo& g);
// One damped-Jacobi sweep x_out = x + omega D^{-1} (f - A x).
template <typename T>
void launch_jacobi(const Geo& g, const Coef<T>& cf, const T* w, const T* f, const T* x, T* xout,
                   double omega, bool zero_init, cudaStream_t st);
// coarse f = average over the children of (f - A x) on the fine level
template <typename T>
void launch_restrict_residual(const Geo& fine, const Coef<T>& cf, const T* f, const T* x,
                             const Geo& coarse, const int fac[3], T* fc, cudaStream_t st);
// FP32 V-cycle with FP16 storage of the (unscaled) level-0 coefficients:
// the colour pass and the residual restriction of the finest level.
void launch_rbgs_h(const Geo& g, const __half* const b[3], float scale, const float* f, float* x,
                   int color, double omega, bool zero_init, cudaStream_t st, int k0 = 0, int k1 = -1);
void launch_restrict_residual_h(const Geo& fine, const __half* const b[3], float scale, const float* f,
                                const float* x, const Geo& coarse, const int fac[3], float* fc,
                                cudaStream_t st);
void launch_convert_beta_half(const Geo& g, const double* const b64[3], __half* const out[3],
                              cudaStream_t st);
// x_fine += x_coarse[parent]
template <typename T>
void launch_prolong_add(const Geo& fine, const Geo& coarse, const int fac[3], const T* xc,
                        T* x, cudaStream_t st);

// ------------------------------------- level 0 rebuilt from the cell densities ---
// rh: FP32 half-densities rho/2 of the finest level (Eq. muH); the kernels
// form beta_f = 1/(rh_L + rh_R) in registers and apply 1/h^2 themselves.
// The FP32 vectors of level 0 (x and f of the smoother, d and q of the inner
// CG, r32 and e of the refinement) are in the colour-split layout: each row
// holds its cells of colour (i+j+k) even in order of i, then the odd ones.
// even nx, ny, nz and 32-bit offsets
bool rho0_fits(const Geo& g);
// tiles: 2 = the TMA-staged plane kernel (stage.cu) where rho0_stage_fits,
// else 1 = the register plane-tile kernels where nx/2 is even, else (0) the
// z-column kernels.  The staged and plane-tile zero pass (zero_init) writes
// the updated colour only; the pass of the other colour that follows it must
// be launched with own_zero, which takes that colour as zero instead of
// reading it.  The z-column kernels write both colours on the zero pass and
// ignore own_zero.  fail: a word the staged kernel sets when one of its
// bounded waits gives up (may be null for the other kernels).
// rh16 (may be null): rho/2 in FP16, read instead of rh by the register
// plane-tile pass (tiles == 1)
void launch_rbgs_rho(const Geo& g, const float* rh, double h, const float* f, float* x, int color,
                     double omega, bool zero_init, cudaStream_t st, int k0 = 0, int k1 = -1, int tiles = 1,
                     bool own_zero = false, unsigned* fail = nullptr, const __half* rh16 = nullptr,
                     bool rev = false);
// whether launch_rbgs_rho runs a plane kernel (staged or register tiles) on this grid
bool rho0_tile_pass(const Geo& g, int tiles);
// the staged colour pass (stage.cu): nx a multiple of 8, ny of its tile height
bool rho0_stage_fits(const Geo& g);
cudaError_t launch_rbgs_rho_stage(const Geo& g, const float* rh, double h, const float* f, float* x, int color,
                                  double omega, bool zero_init, bool own_zero, int k0, int k1, unsigned* fail,
                                  cudaStream_t st);
// q = A d; partials (d . q); returns the number of blocks
int64_t launch_matvec_rho(const Geo& g, const float* rh, double h, const float* d, float* q,
                          double* partials, cudaStream_t st, FinSpec fin = no_fin(), bool tiles = true, bool rev = false);
// the plane-tile product with the flexible CG's direction update fused in:
// dnew = z + beta d (beta from s) and q = A dnew, d . q partials as above
// (dnew must not alias z or d); only where rho0_product_fuses.  e (may be
// null): the previous iteration's solution update e += alpha d rides along
// (alpha from s, read before this launch's finalize replaces it; emem false:
// e taken as 0, not read)
bool rho0_product_fuses(const Geo& g, bool tiles);
int64_t launch_matvec_rho_xpby(const Geo& g, const float* rh, double h, const float* z, const float* d, float* dnew,
                               float* q, const Scal* s, double* partials, cudaStream_t st, FinSpec fin, bool rev = false,
                               float* e = nullptr, bool emem = true);
int64_t rho0_matvec_blocks(const Geo& g);
// coarse f = mean over the 2x2x2 children of (f - A x); coarse = every axis halved
void launch_restrict_rho(const Geo& g, const float* rh, double h, const float* f, const float* x,
                         const Geo& coarse, float* fc, cudaStream_t st, bool tiles = true,
                         const __half* rh16 = nullptr, bool rev = false);
// x += P xc (piecewise constant) onto the split level 0 from the level with every axis halved
void launch_prolong_split(const Geo& fine, const Geo& coarse, const float* xc, float* x, cudaStream_t st, bool rev = false);
// scaled FP32 coefficients of the level with every axis halved; out16 (may be
// null): FP16 copies of the sums of the four fine faces' coefficients times s16
// (the FP32 coefficient is that sum times 1/(16 h^2))
void launch_coarse_beta_rho(const Geo& fine, const float* rh, double h, const Geo& coarse, float* out[3],
                            cudaStream_t st, __half* const out16[3] = nullptr, float s16 = 1.f);

// FP64 refinement step of the mixed form on the finest level, A d in
// double-float from the rho/2 pairs rh2: x += 2^-a e, r_new = r_old - A 2^-a e,
// r32 = 2^b r_new (2^a: s->scale, 2^b from s->rinf), norms (FIN_REFINE fused);
// e and r32 in the colour-split layout.  emem false: e taken as 0 (not read);
// dpend (may be null): the inner solve's last update e += alpha dpend (alpha
// from s) applied first
void launch_refine_rho(const Geo& g, const float2* rh2, double h, const float* e, const double* r_old,
                       double* r_new, double* x, float* r32, Scal* s, double* partials, cudaStream_t st, bool rev = false,
                       bool emem = true, const float* dpend = nullptr);

// ------------------------------------------------ single-launch V-cycle tail ---
// One level of the tail: coefficients (scaled by `scale`), inverse diagonal
// (FP64 V-cycles; null: recomputed), solution and right-hand side, and the
// coarsening factors from the level above.
template <typename T>
struct TailLevel {
    Geo g;
    int fac[3];
    // multipliers of the divisions by nx, ny and the pairs per row (nx + 1)/2:
    // t / n = umulhi(t, m) for t, n < 2^16 with m = ceil(2^32 / n) (n > 1)
    unsigned mx, my, mp;
    T scale;
    const T* bx;
    const T* by;
    const T* bz;
    const T* w;
    T* x;
    T* f;
};
constexpr int kMaxTail = 16;         // levels in one tail launch
constexpr int kMaxDenseCells = 128;  // cells of a dense coarsest level
// The V-cycle from levels[0] (its f already restricted from above) down to
// the dense coarsest levels[n-1] (inverse Minv) and back: one block.
template <typename T>
void launch_tail_vcycle(const TailLevel<T>* levels, int n, const double* Minv, double omega, int nu1,
                        int nu2, bool use_w, cudaStream_t st);

// ------------------------------------------------------------ Krylov ------
// r = f - A x (FP64), optional r32 = scale * r; partials (||r||^2, max|r|, nonfinite).
// zero_ok: x is the initial guess whose max |x| the prologue stored in s->xmax;
// when that is 0 the kernel copies r = f instead of applying A.  split: r32
// in the colour-split layout of level 0 (nx even).
int64_t launch_residual64(const Geo& g, const Coef<double>& cf, const double* f, const double* x,
                          double* r64, float* r32, const Scal* s, double* partials, bool zero_ok,
                          cudaStream_t st, FinSpec fin = no_fin(), bool split = false);
// q = A d; partials (d . q)
template <typename T>
int64_t launch_matvec_dot(const Geo& g, const Coef<T>& cf, const T* d, T* q, double* partials,
                          cudaStream_t st, FinSpec fin = no_fin());
// x += alpha d; r -= alpha q; partials (||r||^2, max|r|, nonfinite)
template <typename T>
int64_t launch_update_xr(int64_t n, const Scal* s, const T* d, const T* q, T* x, T* r,
                         double* partials, cudaStream_t st, FinSpec fin = no_fin(), bool rev = false);
// r -= alpha q and the partials of launch_update_xr (x's update left to the caller)
template <typename T>
int64_t launch_update_r(int64_t n, const Scal* s, const T* q, T* r, double* partials, cudaStream_t st,
                        FinSpec fin = no_fin(), bool rev = false);
// partials (a . b, a . c)  (c may be null -> 0); fin: fused second stage
template <typename T>
int64_t launch_dot2(int64_t n, const T* a, const T* b, const T* c, double* partials,
                    cudaStream_t st, FinSpec fin = no_fin(), bool rev = false);
// d = z + beta d
template <typename T>
void launch_xpby(int64_t n, const Scal* s, const T* z, T* d, cudaStream_t st);
// x64 += e32 * inv_scale
void launch_accumulate(int64_t n, const Scal* s, const float* e, double* x, cudaStream_t st);

// ------------------------------------------------------------ self-check ---
// counts disagreements of the integer conversions and the FP64 reciprocal
// with the hardware instructions on n values (see paris_check_arithmetic)
void launch_check_arithmetic(const double* v, int64_t n, int shift, unsigned long long* bad,
                             cudaStream_t st);

// ------------------------------------------------------------ adjoint -----
// out = D (B g) (walls carry no flux); partials (sum, max|out|, nonfinite)
int64_t launch_weighted_div(const Geo& g, const double* bx, const double* by, const double* bz,
                            const double* gx, const double* gy, const double* gz, double inv_h,
                            double* out, double* partials, cudaStream_t st);
// dLoss/du* = g - G q and dLoss/dbeta = dt (G p)(G q - g) on non-wall faces
void launch_adjoint_faces(const Geo& g, const double* p, const double* q, double inv_h, double dt,
                          const double* gx, const double* gy, const double* gz, double* usx,
                          double* usy, double* usz, double* bbx, double* bby, double* bbz,
                          cudaStream_t st);
// dLoss/dC from dLoss/dbeta through beta = 2/(rho_L + rho_R)
void launch_face_coeffs_adjoint(const Geo& g, double rho1, double rho2, const double* bx,
                                const double* by, const double* bz, const double* gbx,
                                const double* gby, const double* gbz, double* gC, cudaStream_t st);

}  // namespace paris
