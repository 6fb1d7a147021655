// CUDA kernels of the one-fluid pressure projection (sm_103a).
//
// Paper references: PARIS, arXiv 2012.11744.  Eq. muH (one-fluid density),
// Eqs. cont2/incompdisc3 (divergence on the staggered grid), Eq. poisson and
// the A1..A8 system form with its over-relaxed red-black Gauss-Seidel update
// (Eq. eq:beta_pressure, Sec. 3.7.1), the V-cycle of Sec. 3.7.3, the Jacobi
// iteration of Sec. 3.7.4, the link-flag coefficient zeroing at walls
// (Sec. 3.8) and the velocity correction Eq. fotm.
//
// Stencil kernels work in the SPD form A = -L, A x = f with f = -b:
//   (A x)_c = scale * sum_f beta_f (x_c - x_nb),
// i.e. the paper's A7 p - sum A_nb p_nb with A_nb = beta_f scale.
#include <math.h>

#include <atomic>
#include <cstdio>

#include "kernels.cuh"

namespace paris {

namespace {

constexpr int kTX = 32, kTY = 8;  // 2-D tile of the stencil kernels (x fastest)
// rows per block of the colour passes of the face-array levels (rbgs_kernel,
// rbgs4_kernel), by precision: small blocks schedule at finer grain; the
// FP64 step measured 33.6 ms with two rows against 35.9 with eight, the
// mixed one 8.84 ms with four against 8.87 (and 8.92 with two)
#ifndef PARIS_PASS_TY32
#define PARIS_PASS_TY32 4
#endif
#ifndef PARIS_PASS_TY64
#define PARIS_PASS_TY64 2
#endif
template <typename T>
__host__ __device__ constexpr int pass_rows() {
    return sizeof(T) == 8 ? PARIS_PASS_TY64 : PARIS_PASS_TY32;
}
constexpr int kZ = 8;             // cells per thread along z in reducing stencil kernels

// Element-wise grid-stride loop over [0, n).
#define PARIS_EW_FOR(c, n)                                                           \
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < (n);        \
         c += (int64_t)gridDim.x * blockDim.x)

// 16-byte vectors for the streaming kernels: a thread moves 16 bytes of
// each array per load (float4 / double2), so enough bytes are in flight to
// cover the HBM latency with the capped grid.
template <typename T>
struct V16;
template <>
struct V16<float> {
    using type = float4;
    static constexpr int n = 4;
};
template <>
struct V16<double> {
    using type = double2;
    static constexpr int n = 2;
};

// Vector part [0, n/W) of a grid-stride loop, then the scalar tail.
#define PARIS_VEC_FOR(i, nvec)                                                        \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (nvec);      \
         i += (int64_t)gridDim.x * blockDim.x)
#define PARIS_TAIL_FOR(c, start, n)                                                   \
    for (int64_t c = (start) + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < (n); \
         c += (int64_t)gridDim.x * blockDim.x)

// z-loop over [k0, k1)
#define PARIS_ZLOOP(k0, k1, ...)               \
    for (int k = (k0); k < (k1); ++k) {        \
        __VA_ARGS__                            \
    }

inline dim3 tile_grid(const Geo& g, int zper) {
    return dim3((g.nx + kTX - 1) / kTX, (g.ny + kTY - 1) / kTY, (g.nz + zper - 1) / zper);
}

inline int64_t nblocks_of(dim3 gr) { return (int64_t)gr.x * gr.y * gr.z; }

__device__ inline int64_t flat_block() {
    return ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
}

__device__ inline int flat_tid() { return threadIdx.y * blockDim.x + threadIdx.x; }

}  // namespace

static thread_local char g_last_cuda_error[256] = "no CUDA error recorded";
void paris_internal_note_cuda_error(cudaError_t e) {
    snprintf(g_last_cuda_error, sizeof g_last_cuda_error, "%s: %s", cudaGetErrorName(e),
             cudaGetErrorString(e));
}
const char* last_cuda_error() { return g_last_cuda_error; }

static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

// true when every (non-null) pointer is 16-byte aligned: vector loads allowed
inline bool aligned16(const void* a, const void* b = nullptr, const void* c = nullptr,
                      const void* d = nullptr) {
    auto ok = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
    return ok(a) && ok(b) && ok(c) && ok(d);
}

// 32-bit offsets suffice for every array of the level
inline bool fits_i32(const Geo& g) {
    const int64_t big = ((int64_t)1 << 31) - 1;
    return g.nface(0) < big && g.nface(1) < big && g.nface(2) < big;
}

int device_sms() {
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        return 1;
    }
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
        cudaGetLastError();
        return 1;
    }
    cache[dev].store(n, std::memory_order_relaxed);
    return n;
}

int elementwise_blocks(int64_t n) {
    int64_t b = (n + kRedThreads - 1) / kRedThreads;
    // 256-thread blocks per SM of the streaming kernels: with four 16-byte loads
    // per array in flight per thread, 3 blocks per SM saturate the memory and keep
    // the last-block reductions short (the 256^3 step: 9.86 ms at 8, 9.69 at 3)
#ifndef PARIS_EW_PER_SM
#define PARIS_EW_PER_SM 3
#endif
    const int64_t cap = (int64_t)device_sms() * PARIS_EW_PER_SM;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

int64_t max_reduce_blocks(const Geo& g) {
    const int64_t tiles = nblocks_of(tile_grid(g, kZ));
    const int64_t ew = elementwise_blocks(g.ncell());
    return tiles > ew ? tiles : ew;
}

// ---------------------------------------------------------------- finalize ---

// Deterministic second stage of every reduction: one CTA folds the block
// partials in a fixed order, then thread 0 applies the scalar update `mode`.
__global__ void finalize_kernel(const double* __restrict__ partials, int64_t nblocks, int nv,
                                int maxmask, Scal* s, int mode, double param) {
    finalize_block(partials, nblocks, nv, maxmask, s, mode, param, threadIdx.x);
}

void finalize(const double* partials, int64_t nblocks, int nv, int maxmask, Scal* s, int mode,
              double param, cudaStream_t st) {
    finalize_kernel<<<1, kRedThreads, 0, st>>>(partials, nblocks, nv, maxmask, s, mode, param);
    count_launch();
}

// ------------------------------------------------------- face coefficients ---

// 1/s for s > 0 without an FP64 division and without FP64<->FP32
// conversions (both run at the FP64 rate, 1/64 of the FP32 rate on this
// GPU): an FP32 estimate is formed from the leading bits of s by re-biasing
// the exponent in integer arithmetic (20 of the 52 fraction bits kept, so
// the estimate is within 2^-20 of s), inverted with the FP32 approximate
// reciprocal (1 ulp), re-biased back into an FP64 y0 with |1 - s y0| < 2^-19.
// One third-order Newton-Raphson step y0 (1 + e + e^2), e = 1 - s y0,
// leaves a truncation error e^3 < 2^-57 relative, below half an ulp, so the
// result is within one ulp of the correctly rounded 1/s.  Values of s
// outside the exponent window [2^-123, 2^117) (or s <= 0, NaN) take the
// FP64 division.
__device__ inline double recip64(double s) {
    const int hi = __double2hiint(s);
    if (hi < (900 << 20) || hi >= (1140 << 20)) return 1.0 / s;
    const float sf = __int_as_float((hi - (896 << 20)) << 3);
    float yf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(sf));
    const unsigned yb = (unsigned)__float_as_int(yf);
    const double y0 = __hiloint2double((int)((yb >> 3) + (896u << 20)), (int)(yb << 29));
    const double e = fma(-s, y0, 1.0);
    return fma(y0, fma(e, e, e), y0);
}

constexpr int kFSeg = 16;  // planes per thread of the face-coefficient kernel

// Eq. muH: rho = rho1 C + rho2 (1 - C); beta_f = 1/rho_f with rho_f the mean
// of the two cells (the paper's "interpolation of 1/rho" read as the mean of
// rho, then inverted); wall faces 0 (Sec. 3.8).  Computed as rh = rho/2 from
// rho1/2 and rho2/2 (exact scalings), beta_f = 1/(rh_L + rh_R).
// A thread owns the column (i, j) over a segment of planes and writes the -
// face of each axis (the last cell of a wall axis also writes the + wall
// face).  Each cell's rh is evaluated once: the z-neighbour's is carried in
// a register, the x- and y-neighbours' come through a shared-memory tile
// whose halo row and column are evaluated by one warp each.  Optionally
// writes the FP32 copy of rho/2 that the mixed solve's finest level reads.
//
// With FORCE (the predictor's capillary and gravity forcing, Eq.
// nonconspredictedvel with the CSF term of Eq. csf2), the same pass also
// writes u* = u^n + tau a_f in place on every face it owns, with
//   a_f = g_a - (sigma/h) kappa_f (C_R - C_L) beta_f,  kappa_f = (kappa_L + kappa_R)/2,
// beta_f the coefficient it has just formed (so a constant kappa gives
// beta_f times a face gradient of -sigma kappa C: exactly what the projection
// removes); wall faces get u* = 0.  C and kappa of the neighbours come
// through shared-memory tiles like rh.
struct ForceArgs {
    const double* kappa;  // cells; null: kappa = 0
    double s_over_h;      // sigma / h
    double g[3];          // gravity (acceleration) per axis
    double tau;           // time step of the predictor
    double* u[3];         // face arrays: in u^n, out u*
};

template <bool FORCE>
__global__ void __launch_bounds__(kTX* kTY) face_coeffs_kernel(Geo g, const double* __restrict__ C,
                                                              double r1h, double r2h,
                                                              double* __restrict__ bx,
                                                              double* __restrict__ by,
                                                              double* __restrict__ bz,
                                                              float* __restrict__ rh32,
                                                              float2* __restrict__ rh2, ForceArgs fa) {
    __shared__ double sh[2][kTY + 1][kTX + 1];  // [plane parity][1 + row][1 + column]
    __shared__ double shc[FORCE ? 2 : 1][kTY + 1][kTX + 1];  // C (FORCE)
    __shared__ double shk[FORCE ? 2 : 1][kTY + 1][kTX + 1];  // kappa (FORCE)
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int i = blockIdx.x * kTX + tx, j = blockIdx.y * kTY + ty;
    const bool in = i < nx && j < ny;
    const int ic = min(i, nx - 1), jc = min(j, ny - 1);  // idle threads shadow a cell
    const int kb = blockIdx.z * kFSeg, ke = min(kb + kFSeg, nz);
    const int64_t pl = (int64_t)nx * ny;
    auto rho = [&](double c) { return fma(r1h, c, r2h * (1.0 - c)); };
    auto kap = [&](int64_t c) { return fa.kappa ? fa.kappa[c] : 0.0; };
    // halo cells: row j0-1 (warp 0) and column i0-1 (lanes 0..7 of warp 1)
    const int i0 = blockIdx.x * kTX, j0 = blockIdx.y * kTY;
    const int hx = i0 > 0 ? i0 - 1 : nx - 1;  // periodic wrap (walls: beta 0, value unused)
    const int hy = j0 > 0 ? j0 - 1 : ny - 1;
    const int hrow = min(j0 + tx, ny - 1);       // row of the column-halo cell of lane tx
    const int hcol = min(i0 + tx, nx - 1);       // column of the row-halo cell of lane tx
    const bool xw = g.wx && i == 0, yw = g.wy && j == 0;
    const int64_t czm_at = (int64_t)(kb > 0 ? kb - 1 : nz - 1) * pl + (int64_t)jc * nx + ic;
    double czm = C[czm_at];
    double rzm = rho(czm);
    double kzm = FORCE ? kap(czm_at) : 0.0;
    for (int k = kb; k < ke; ++k) {
        const int64_t plane = (int64_t)k * pl;
        const int64_t c = plane + (int64_t)jc * nx + ic;
        const double cc = C[c];
        const double rc = rho(cc);
        const int b = k & 1;
        sh[b][ty + 1][tx + 1] = rc;
        const int64_t crow = plane + (int64_t)hy * nx + hcol, ccol = plane + (int64_t)hrow * nx + hx;
        double kc = 0.0;
        if (ty == 0) {
            const double ch = C[crow];
            sh[b][0][tx + 1] = rho(ch);
            if (FORCE) {
                shc[b][0][tx + 1] = ch;
                shk[b][0][tx + 1] = kap(crow);
            }
        }
        if (ty == 1 && tx < kTY) {
            const double ch = C[ccol];
            sh[b][tx + 1][0] = rho(ch);
            if (FORCE) {
                shc[b][tx + 1][0] = ch;
                shk[b][tx + 1][0] = kap(ccol);
            }
        }
        if (FORCE) {
            kc = kap(c);
            shc[b][ty + 1][tx + 1] = cc;
            shk[b][ty + 1][tx + 1] = kc;
        }
        __syncthreads();
        const double rxm = sh[b][ty + 1][tx], rym = sh[b][ty][tx + 1];
        if (in) {
            const double bxv = xw ? 0.0 : recip64(rxm + rc);
            const double byv = yw ? 0.0 : recip64(rym + rc);
            const bool zw = g.wz && k == 0;
            const double bzv = zw ? 0.0 : recip64(rzm + rc);
            const int64_t fxi = g.fx(i, j, k), fyi = g.fy(i, j, k), fzi = g.fz(i, j, k);
            bx[fxi] = bxv;
            by[fyi] = byv;
            bz[fzi] = bzv;
            if (g.wx && i == nx - 1) bx[g.fx(nx, j, k)] = 0.0;
            if (g.wy && j == ny - 1) by[g.fy(i, ny, k)] = 0.0;
            if (g.wz && k == nz - 1) bz[g.fz(i, j, nz)] = 0.0;
            if (FORCE) {
                // u*_f = u^n_f + tau (g_a - (sigma/h) kappa_f (C_R - C_L) beta_f); 0 on walls
                auto star = [&](double* u, int64_t f, bool wall, double cl, double kl, double bf, double ga) {
                    if (wall) {
                        u[f] = 0.0;
                        return;
                    }
                    const double kf = 0.5 * (kl + kc);
                    const double a = ga - fa.s_over_h * kf * (cc - cl) * bf;
                    u[f] = fma(fa.tau, a, u[f]);
                };
                star(fa.u[0], fxi, xw, shc[b][ty + 1][tx], shk[b][ty + 1][tx], bxv, fa.g[0]);
                star(fa.u[1], fyi, yw, shc[b][ty][tx + 1], shk[b][ty][tx + 1], byv, fa.g[1]);
                star(fa.u[2], fzi, zw, czm, kzm, bzv, fa.g[2]);
                if (g.wx && i == nx - 1) fa.u[0][g.fx(nx, j, k)] = 0.0;
                if (g.wy && j == ny - 1) fa.u[1][g.fy(i, ny, k)] = 0.0;
                if (g.wz && k == nz - 1) fa.u[2][g.fz(i, j, nz)] = 0.0;
            }
            if (rh32) {
                const float hi = d2f_scaled(rc, 0);
                rh32[c] = hi;
                // the remainder is exact in FP64; its FP32 rounding completes the pair
                if (rh2) rh2[c] = make_float2(hi, d2f_scaled(rc - f2d_scaled(hi, 0), 0));
            }
        }
        rzm = rc;
        if (FORCE) {
            czm = cc;
            kzm = kc;
        }
    }
}

// a + b = s.x + s.y exactly (Knuth's two-sum, FP32)
__device__ __forceinline__ float2 two_sum_f(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp)));
}

// 1/(a + b) for two (hi, lo) FP32 pairs in FP32 arithmetic, returned in FP64:
// the pair sum S (leading part by two-sum, the rest added), y0 the
// approximate reciprocal of its leading part (1 ulp), t = 1 - S y0 (to about
// 2^-47), 1/S = y0 (1 + t + t^2 + ...) kept to second order: y0 + y0 (t + t^2)
// as an FP64 sum of two FP32 numbers, about 46 significant bits.
__device__ __forceinline__ double recip_pair_sum(float2 a, float2 b) {
    const float2 s = two_sum_f(a.x, b.x);
    const float slo = __fadd_rn(s.y, __fadd_rn(a.y, b.y));
    float y0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(s.x));
    float t = __fmaf_rn(-s.x, y0, 1.0f);
    t = __fmaf_rn(-slo, y0, t);
    const float blo = __fmul_rn(y0, __fmaf_rn(t, t, t));
    return f2d_scaled(y0, 0) + f2d_scaled(blo, 0);
}

// The face coefficients of the mixed form's projection step, with the FP64
// pipe (1/64 of the FP32 rate on this GPU) used for three operations per
// cell instead of about seventeen: rh = rho/2 = rh2 + C (rh1 - rh2) by one
// FMA, its (hi, lo) FP32 split (one FP64 subtraction), and per face beta_f =
// 1/(rh_L + rh_R) from the two pairs in FP32 arithmetic (recip_pair_sum) with
// one FP64 addition.  beta_f is then within about 2^-46 of 1/rho_f (the exact
// form, face_coeffs_kernel, is within one ulp): the operator the mixed form's
// double-float refinement step already applies.  Same tiling as
// face_coeffs_kernel; writes rh32 and rh2 too.
__global__ void __launch_bounds__(kTX* kTY) face_coeffs_fast_kernel(Geo g, const double* __restrict__ C,
                                                                   double d12h, double r2h,
                                                                   double* __restrict__ bx,
                                                                   double* __restrict__ by,
                                                                   double* __restrict__ bz,
                                                                   float* __restrict__ rh32,
                                                                   float2* __restrict__ rh2,
                                                                   __half* __restrict__ rh16) {
    __shared__ float2 sh[2][kTY + 1][kTX + 1];  // [plane parity][1 + row][1 + column]
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int i = blockIdx.x * kTX + tx, j = blockIdx.y * kTY + ty;
    const bool in = i < nx && j < ny;
    const int ic = min(i, nx - 1), jc = min(j, ny - 1);  // idle threads shadow a cell
    const int kb = blockIdx.z * kFSeg, ke = min(kb + kFSeg, nz);
    const int64_t pl = (int64_t)nx * ny;
    auto pair = [&](double c) {
        const double rh = fma(d12h, c, r2h);
        const float hi = d2f_scaled(rh, 0);
        return make_float2(hi, d2f_scaled(rh - f2d_scaled(hi, 0), 0));
    };
    const int i0 = blockIdx.x * kTX, j0 = blockIdx.y * kTY;
    const int hx = i0 > 0 ? i0 - 1 : nx - 1;  // periodic wrap (walls: beta 0, value unused)
    const int hy = j0 > 0 ? j0 - 1 : ny - 1;
    const int hrow = min(j0 + tx, ny - 1);
    const int hcol = min(i0 + tx, nx - 1);
    const bool xw = g.wx && i == 0, yw = g.wy && j == 0;
    float2 rzm = pair(C[(int64_t)(kb > 0 ? kb - 1 : nz - 1) * pl + (int64_t)jc * nx + ic]);
    for (int k = kb; k < ke; ++k) {
        const int64_t plane = (int64_t)k * pl;
        const int64_t c = plane + (int64_t)jc * nx + ic;
        const float2 rc = pair(C[c]);
        const int b = k & 1;
        sh[b][ty + 1][tx + 1] = rc;
        if (ty == 0) sh[b][0][tx + 1] = pair(C[plane + (int64_t)hy * nx + hcol]);
        if (ty == 1 && tx < kTY) sh[b][tx + 1][0] = pair(C[plane + (int64_t)hrow * nx + hx]);
        __syncthreads();
        if (in) {
            const bool zw = g.wz && k == 0;
            bx[g.fx(i, j, k)] = xw ? 0.0 : recip_pair_sum(sh[b][ty + 1][tx], rc);
            by[g.fy(i, j, k)] = yw ? 0.0 : recip_pair_sum(sh[b][ty][tx + 1], rc);
            bz[g.fz(i, j, k)] = zw ? 0.0 : recip_pair_sum(rzm, rc);
            if (g.wx && i == nx - 1) bx[g.fx(nx, j, k)] = 0.0;
            if (g.wy && j == ny - 1) by[g.fy(i, ny, k)] = 0.0;
            if (g.wz && k == nz - 1) bz[g.fz(i, j, nz)] = 0.0;
            rh32[c] = rc.x;
            rh2[c] = rc;
            if (rh16) rh16[c] = __float2half_rn(rc.x);
        }
        rzm = rc;
    }
}

void launch_face_coeffs_fast(const Geo& g, const double* C, double rho1, double rho2, double* bx, double* by,
                             double* bz, float* rh32, float2* rh2, __half* rh16, cudaStream_t st) {
    dim3 gr((g.nx + kTX - 1) / kTX, (g.ny + kTY - 1) / kTY, (g.nz + kFSeg - 1) / kFSeg);
    face_coeffs_fast_kernel<<<gr, dim3(kTX, kTY), 0, st>>>(g, C, 0.5 * rho1 - 0.5 * rho2, 0.5 * rho2, bx, by, bz,
                                                           rh32, rh2, rh16);
    count_launch();
}

void launch_face_coeffs(const Geo& g, const double* C, double rho1, double rho2, double* bx,
                        double* by, double* bz, float* rh32, float2* rh2, cudaStream_t st,
                        const Forcing* force) {
    dim3 gr((g.nx + kTX - 1) / kTX, (g.ny + kTY - 1) / kTY, (g.nz + kFSeg - 1) / kFSeg);
    if (force) {
        ForceArgs fa{force->kappa, force->sigma / force->h, {force->g[0], force->g[1], force->g[2]},
                     force->tau, {force->u[0], force->u[1], force->u[2]}};
        face_coeffs_kernel<true><<<gr, dim3(kTX, kTY), 0, st>>>(g, C, 0.5 * rho1, 0.5 * rho2, bx, by, bz, rh32,
                                                                rh2, fa);
    } else {
        face_coeffs_kernel<false><<<gr, dim3(kTX, kTY), 0, st>>>(g, C, 0.5 * rho1, 0.5 * rho2, bx, by, bz, rh32,
                                                                 rh2, ForceArgs{});
    }
    count_launch();
}

// -------------------------------------------------------------- divergence ---

// Sum over the axes of (u_{+face} - u_{-face}) (Eqs. cont2, incompdisc3),
// wall faces carrying no flux; times 1/(h dt).
__device__ inline double cell_div(const Geo& g, const double* __restrict__ u,
                                  const double* __restrict__ v, const double* __restrict__ w,
                                  int i, int j, int k) {
    AxisNb ax = axis_nb(i, g.nx, g.wx), ay = axis_nb(j, g.ny, g.wy), az = axis_nb(k, g.nz, g.wz);
    double up = ax.wp ? 0.0 : u[g.fx(ax.fp, j, k)];
    double um = ax.wm ? 0.0 : u[g.fx(i, j, k)];
    double vp = ay.wp ? 0.0 : v[g.fy(i, ay.fp, k)];
    double vm = ay.wm ? 0.0 : v[g.fy(i, j, k)];
    double wp = az.wp ? 0.0 : w[g.fz(i, j, az.fp)];
    double wm = az.wm ? 0.0 : w[g.fz(i, j, k)];
    return ((up - um) + (vp - vm)) + (wp - wm);
}

__global__ void __launch_bounds__(kTX* kTY) divergence_kernel(Geo g, const double* __restrict__ u,
                                                              const double* __restrict__ v,
                                                              const double* __restrict__ w,
                                                              double inv_hdt,
                                                              double* __restrict__ rhs,
                                                              double* partials, FinSpec fin) {
    const int i = blockIdx.x * kTX + threadIdx.x;
    const int j = blockIdx.y * kTY + threadIdx.y;
    double sum = 0.0;
    unsigned long long bmax_k = 0;
    unsigned nf = 0;
    if (i < g.nx && j < g.ny) {
        const int k0 = blockIdx.z * kZ, k1 = min(k0 + kZ, g.nz);
        PARIS_ZLOOP(k0, k1, {
            const double b = cell_div(g, u, v, w, i, j, k) * inv_hdt;
            rhs[g.cidx(i, j, k)] = b;
            sum += b;
            const unsigned long long kb = abs_key(b);
            bmax_k = kb > bmax_k ? kb : bmax_k;
            nf += key_nonfinite(kb);
        })
    }
    block_reduce_skc<double>(sum, bmax_k, nf, partials, flat_block(), flat_tid());
    finalize_last_block(partials, (int64_t)gridDim.x * gridDim.y * gridDim.z, fin, flat_tid());
}

int64_t launch_divergence(const Geo& g, const double* u, const double* v, const double* w,
                          double inv_hdt, double* rhs, double* partials, cudaStream_t st, FinSpec fin) {
    dim3 gr = tile_grid(g, kZ);
    divergence_kernel<<<gr, dim3(kTX, kTY), 0, st>>>(g, u, v, w, inv_hdt, rhs, partials, fin);
    count_launch();
    return nblocks_of(gr);
}

__global__ void __launch_bounds__(kTX* kTY) max_div_kernel(Geo g, const double* __restrict__ u,
                                                           const double* __restrict__ v,
                                                           const double* __restrict__ w,
                                                           double inv_h, double* partials) {
    const int i = blockIdx.x * kTX + threadIdx.x;
    const int j = blockIdx.y * kTY + threadIdx.y;
    unsigned long long dmax_k = 0;
    if (i < g.nx && j < g.ny) {
        const int k0 = blockIdx.z * kZ, k1 = min(k0 + kZ, g.nz);
        PARIS_ZLOOP(k0, k1, {
            const unsigned long long kd = abs_key(cell_div(g, u, v, w, i, j, k));
            dmax_k = kd > dmax_k ? kd : dmax_k;
        })
    }
    // max |div| h^-1 = h^-1 max |div| (h > 0)
    double acc[1] = {key_value(dmax_k) * inv_h};
    const int op[1] = {1};
    block_reduce_store<1>(acc, op, partials, flat_block(), flat_tid());
}

int64_t launch_max_divergence(const Geo& g, const double* u, const double* v, const double* w,
                              double inv_h, double* partials, cudaStream_t st) {
    dim3 gr = tile_grid(g, kZ);
    max_div_kernel<<<gr, dim3(kTX, kTY), 0, st>>>(g, u, v, w, inv_h, partials);
    count_launch();
    return nblocks_of(gr);
}

// f = -(rhs - mean_b): the right-hand side of the SPD system A p = f; with
// solid cells (solid[c] == 0, Sec. 3.8) f = 0 there, each such cell being a
// null direction of the masked operator on its own.
__global__ void make_rhs_kernel(int64_t n, const double* __restrict__ rhs, const Scal* s,
                                double* __restrict__ f, const double* __restrict__ x0,
                                double* partials, FinSpec fin, const unsigned char* __restrict__ solid) {
    const double mb = s->mean_b;
    double l2 = 0.0;
    unsigned long long fmax_k = 0, xmax_k = 0;
    unsigned nf = 0;
    PARIS_EW_FOR(c, n) {
        const double t = (solid && !solid[c]) ? 0.0 : -(rhs[c] - mb);
        f[c] = t;
        l2 = fma(t, t, l2);
        const unsigned long long k = abs_key(t);
        fmax_k = k > fmax_k ? k : fmax_k;
        nf += key_nonfinite(k);
        if (x0) {
            const unsigned long long kx = abs_key(x0[c]);
            xmax_k = kx > xmax_k ? kx : xmax_k;
        }
    }
    // without an initial guess the fourth value reads "not known to be zero"
    double acc[4] = {l2, key_value(fmax_k), (double)nf, x0 ? key_value(xmax_k) : 1.0};
    const int op[4] = {0, 1, 0, 1};
    block_reduce_store<4>(acc, op, partials, blockIdx.x, threadIdx.x);
    finalize_last_block(partials, gridDim.x, fin, threadIdx.x);
}

int64_t launch_make_rhs(int64_t n, const double* rhs, const Scal* s, double* f, const double* x0,
                        double* partials, cudaStream_t st, FinSpec fin, const unsigned char* solid) {
    int nb = elementwise_blocks(n);
    make_rhs_kernel<<<nb, kRedThreads, 0, st>>>(n, rhs, s, f, x0, partials, fin, solid);
    count_launch();
    return nb;
}

__global__ void sub_mean_kernel(int64_t n, double* __restrict__ x, const Scal* s) {
    const double m = s->red[0] / (double)n;
    PARIS_EW_FOR(c, n)
        x[c] -= m;
}

void launch_sub_mean(int64_t n, double* x, const Scal* s, cudaStream_t st) {
    sub_mean_kernel<<<elementwise_blocks(n), kRedThreads, 0, st>>>(n, x, s);
    count_launch();
}

__global__ void sum_kernel(int64_t n, const double* __restrict__ x, double* partials) {
    double sum = 0.0;
    unsigned long long xmax_k = 0;
    unsigned nf = 0;
    PARIS_EW_FOR(c, n) {
        const double v = x[c];
        sum += v;
        const unsigned long long k = abs_key(v);
        xmax_k = k > xmax_k ? k : xmax_k;
        nf += key_nonfinite(k);
    }
    block_reduce_skc<double>(sum, xmax_k, nf, partials, blockIdx.x, threadIdx.x);
}

int64_t launch_sum(int64_t n, const double* x, double* partials, cudaStream_t st) {
    int nb = elementwise_blocks(n);
    sum_kernel<<<nb, kRedThreads, 0, st>>>(n, x, partials);
    count_launch();
    return nb;
}

// ------------------------------------------------------ velocity correction ---

// Eq. fotm: u_f -= dt beta_f (p_R - p_L)/h on non-wall faces; wall faces
// blocked to 0 (Sec. 3.8).  Thread per cell, handling its - faces (and the
// + wall face of the last cell of a wall axis).
__global__ void project_kernel(Geo g, const double* __restrict__ bx, const double* __restrict__ by,
                               const double* __restrict__ bz, const double* __restrict__ p,
                               double dt_over_h, double* __restrict__ u, double* __restrict__ v,
                               double* __restrict__ w) {
    const int i = blockIdx.x * kTX + threadIdx.x;
    const int j = blockIdx.y * kTY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const double pc = p[g.cidx(i, j, k)];
    AxisNb ax = axis_nb(i, g.nx, g.wx), ay = axis_nb(j, g.ny, g.wy), az = axis_nb(k, g.nz, g.wz);
    {
        int64_t f = g.fx(i, j, k);
        u[f] = ax.wm ? 0.0 : u[f] - dt_over_h * bx[f] * (pc - p[g.cidx(ax.m, j, k)]);
        if (g.wx && i == g.nx - 1) u[g.fx(g.nx, j, k)] = 0.0;
    }
    {
        int64_t f = g.fy(i, j, k);
        v[f] = ay.wm ? 0.0 : v[f] - dt_over_h * by[f] * (pc - p[g.cidx(i, ay.m, k)]);
        if (g.wy && j == g.ny - 1) v[g.fy(i, g.ny, k)] = 0.0;
    }
    {
        int64_t f = g.fz(i, j, k);
        w[f] = az.wm ? 0.0 : w[f] - dt_over_h * bz[f] * (pc - p[g.cidx(i, j, az.m)]);
        if (g.wz && k == g.nz - 1) w[g.fz(i, j, g.nz)] = 0.0;
    }
}

void launch_project(const Geo& g, const double* bx, const double* by, const double* bz,
                    const double* p, double dt_over_h, double* u, double* v, double* w,
                    cudaStream_t st) {
    dim3 gr((g.nx + kTX - 1) / kTX, (g.ny + kTY - 1) / kTY, g.nz);
    project_kernel<<<gr, dim3(kTX, kTY), 0, st>>>(g, bx, by, bz, p, dt_over_h, u, v, w);
    count_launch();
}

// ------------------------------------------------------------ level set-up ---

// Level-0 coefficient copy in the solver's precision, pre-multiplied by scale.
template <typename T>
__global__ void convert_beta_kernel(int64_t n, const double* __restrict__ b, double scale,
                                    T* __restrict__ out) {
    PARIS_EW_FOR(c, n)
        out[c] = (T)(b[c] * scale);
}

template <typename T>
void launch_convert_beta(const Geo& g, const double* b64[3], double scale, T* out[3],
                         cudaStream_t st) {
    for (int a = 0; a < 3; ++a) {
        int64_t n = g.nface(a);
        convert_beta_kernel<T><<<elementwise_blocks(n), kRedThreads, 0, st>>>(n, b64[a], scale,
                                                                              out[a]);
        count_launch();
    }
}

void launch_convert_scaled(int64_t n, const double* in, double scale, float* out, cudaStream_t st) {
    convert_beta_kernel<float><<<elementwise_blocks(n), kRedThreads, 0, st>>>(n, in, scale, out);
    count_launch();
}

// Rediscretised coarse coefficients (the paper gives no coarsening rule,
// Sec. 3.7.3): a coarse face normal to axis a is covered by the fine faces
// at fine index f_a*I_a along a and f_b*I_b + {0..f_b-1} along the other
// axes b; its coefficient is their mean times (h_fine/h_coarse)^2 along a
// (the arrays hold beta/h_a^2).  Wall faces stay 0.
template <typename T>
__global__ void coarse_beta_kernel(Geo fg, Coef<T> cf, Geo cg, int fa0, int fa1, int fa2,
                                   int axis, double ratio, T* __restrict__ out) {
    const int n0 = cg.nx + (axis == 0 ? cg.wx : 0);
    const int n1 = cg.ny + (axis == 1 ? cg.wy : 0);
    const int n2 = cg.nz + (axis == 2 ? cg.wz : 0);
    const int64_t total = (int64_t)n0 * n1 * n2;
    const int fac[3] = {fa0, fa1, fa2};
    const T* src = axis == 0 ? cf.bx : (axis == 1 ? cf.by : cf.bz);
    const int fn0 = fg.nx + (axis == 0 ? fg.wx : 0);
    const int fn1 = fg.ny + (axis == 1 ? fg.wy : 0);
    PARIS_EW_FOR(t, total) {
        const int I = (int)(t % n0);
        const int J = (int)((t / n0) % n1);
        const int K = (int)(t / ((int64_t)n0 * n1));
        const int C3[3] = {I, J, K};
        int lo[3], cnt[3];
        for (int b = 0; b < 3; ++b) {
            if (b == axis) { lo[b] = C3[b] * fac[b]; cnt[b] = 1; }
            else { lo[b] = C3[b] * fac[b]; cnt[b] = fac[b]; }
        }
        double sum = 0.0;
        for (int dk = 0; dk < cnt[2]; ++dk)
            for (int dj = 0; dj < cnt[1]; ++dj)
                for (int di = 0; di < cnt[0]; ++di) {
                    int64_t fi = ((int64_t)(lo[2] + dk) * fn1 + (lo[1] + dj)) * fn0 + (lo[0] + di);
                    sum += (double)src[fi];
                }
        double mean = sum / (double)(cnt[0] * cnt[1] * cnt[2]);
        out[t] = (T)(mean * ratio * (double)cf.scale);
    }
}

template <typename T>
void launch_coarse_beta(const Geo& fine, const Coef<T>& cf, const Geo& coarse, const int f[3],
                        const double hc2_over_hf2[3], T* out[3], cudaStream_t st) {
    for (int a = 0; a < 3; ++a) {
        int64_t n = coarse.nface(a);
        coarse_beta_kernel<T><<<elementwise_blocks(n), kRedThreads, 0, st>>>(
            fine, cf, coarse, f[0], f[1], f[2], a, 1.0 / hc2_over_hf2[a], out[a]);
        count_launch();
    }
}

// Coarse diagonal excess: the mean over the children of the fine one times
// the fine level's scale (the coarse levels hold absolute coefficients), the
// restriction of the fine equations (an average) applied to sig x with x
// constant over the children.
template <typename T>
__global__ void coarse_sig_kernel(Geo fg, const T* __restrict__ sf, double scale, Geo cg, int fa0, int fa1,
                                  int fa2, T* __restrict__ out) {
    const int64_t total = cg.ncell();
    PARIS_EW_FOR(t, total) {
        const int I = (int)(t % cg.nx);
        const int J = (int)((t / cg.nx) % cg.ny);
        const int K = (int)(t / ((int64_t)cg.nx * cg.ny));
        double sum = 0.0;
        for (int dk = 0; dk < fa2; ++dk)
            for (int dj = 0; dj < fa1; ++dj)
                for (int di = 0; di < fa0; ++di)
                    sum += (double)sf[fg.cidx(I * fa0 + di, J * fa1 + dj, K * fa2 + dk)];
        out[t] = (T)(sum / (double)(fa0 * fa1 * fa2) * scale);
    }
}

template <typename T>
void launch_coarse_sig(const Geo& fine, const T* sig, double scale, const Geo& coarse, const int f[3], T* out,
                       cudaStream_t st) {
    coarse_sig_kernel<T><<<elementwise_blocks(coarse.ncell()), kRedThreads, 0, st>>>(fine, sig, scale, coarse,
                                                                                      f[0], f[1], f[2], out);
    count_launch();
}

// w = 1 / (sum_f beta_f + sig_c) (unscaled inverse diagonal; the smoother
// divides the right-hand side by the level's scale).
template <typename T>
__global__ void inv_diag_kernel(Geo g, Coef<T> cf, T* __restrict__ w) {
    const int i = blockIdx.x * kTX + threadIdx.x;
    const int j = blockIdx.y * kTY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    Stencil<T> s;
    load_stencil(g, cf, i, j, k, s);
    const int64_t c = g.cidx(i, j, k);
    if (cf.sig) {  // the diagonal of a Dirichlet-coupled cell includes its excess
        const T d = (((s.b[0] + s.b[1]) + (s.b[2] + s.b[3])) + (s.b[4] + s.b[5])) + cf.sig[c];
        w[c] = d > T(0) ? rcp_rn(d) : T(0);
    } else {
        w[c] = inv_sum6(s.b);
    }
}

template <typename T>
void launch_inv_diag(const Geo& g, const Coef<T>& cf, T* w, cudaStream_t st) {
    dim3 gr((g.nx + kTX - 1) / kTX, (g.ny + kTY - 1) / kTY, g.nz);
    inv_diag_kernel<T><<<gr, dim3(kTX, kTY), 0, st>>>(g, cf, w);
    count_launch();
}

// Dense inverse of the coarsest operator regularised on its null space:
// (A + a 1 1^T)^{-1} with a = mean(diag)/n, which maps a mean-free f to the
// mean-free solution of A x = f (with a diagonal excess, cf.sig: A^{-1}).  FP64 Gauss-Jordan without pivoting (the
// regularised matrix is SPD) by one CTA of 32 x 32 threads on a copy of the
// matrix in shared memory (n <= 128: at most 129 KB); the elimination step
// maps rows to threadIdx.y and columns to threadIdx.x.
template <typename T>
__global__ void __launch_bounds__(1024) coarse_inverse_kernel(Geo g, Coef<T> cf, double* __restrict__ Mout) {
    extern __shared__ double smem[];
    const int n = (int)g.ncell();
    double* M = smem;         // n x n, row-major
    double* col = smem + n * n;  // column kk before the pivot step
    __shared__ double dsum, piv;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * blockDim.x + tx, nt = blockDim.x * blockDim.y;
    for (int e = tid; e < n * n; e += nt) M[e] = 0.0;
    __syncthreads();
    // each row is assembled by one thread
    for (int c = tid; c < n; c += nt) {
        const int i = c % g.nx, j = (c / g.nx) % g.ny, k = c / (g.nx * g.ny);
        Stencil<T> s;
        load_stencil(g, cf, i, j, k, s);
        for (int q = 0; q < 6; ++q) {
            const double b = (double)s.b[q] * (double)cf.scale;
            M[c * n + c] += b;
            M[c * n + (int)s.nb[q]] -= b;  // a self-neighbour (n = 1) cancels
        }
        if (cf.sig) M[c * n + c] += (double)cf.sig[c] * (double)cf.scale;
    }
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int c = 0; c < n; ++c) t += M[c * n + c];
        dsum = t;
    }
    __syncthreads();
    // a cell with no open face (inside a solid, Sec. 3.8) has a zero row and
    // column: it is decoupled as an identity row and kept out of the
    // regularisation, which then acts on the constants of the other cells
    // (a Dirichlet-coupled operator, cf.sig set, has no null space: no term)
    const double a = cf.sig ? 0.0 : dsum / ((double)n * (double)n);
    for (int e = tid; e < n * n; e += nt) {
        const int r = e / n, cc = e % n;
        const bool ir = M[r * n + r] == 0.0, ic = M[cc * n + cc] == 0.0;
        if (!ir && !ic) M[e] += a;
    }
    __syncthreads();
    for (int c = tid; c < n; c += nt)
        if (M[c * n + c] == 0.0) M[c * n + c] = 1.0;
    __syncthreads();
    for (int kk = 0; kk < n; ++kk) {
        if (tid == 0) piv = 1.0 / M[kk * n + kk];
        for (int r = tid; r < n; r += nt) col[r] = M[r * n + kk];
        __syncthreads();
        for (int c = tid; c < n; c += nt) M[kk * n + c] = (c == kk) ? piv : M[kk * n + c] * piv;
        __syncthreads();
        for (int r = ty; r < n; r += blockDim.y) {
            if (r == kk) continue;
            const double fr = col[r];
            for (int c = tx; c < n; c += blockDim.x)
                M[r * n + c] = (c == kk) ? -fr * piv : fma(-fr, M[kk * n + c], M[r * n + c]);
        }
        __syncthreads();
    }
    for (int e = tid; e < n * n; e += nt) Mout[e] = M[e];
}

template <typename T>
void launch_coarse_inverse(const Geo& g, const Coef<T>& cf, double* inv, cudaStream_t st) {
    const int n = (int)g.ncell();
    const size_t bytes = sizeof(double) * ((size_t)n * n + n);
    static bool opted = false;  // one opt-in per instantiation for more than 48 KB
    if (!opted) {
        cudaFuncSetAttribute(coarse_inverse_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * (128 * 128 + 128)));
        opted = true;
    }
    coarse_inverse_kernel<T><<<1, dim3(32, 32), bytes, st>>>(g, cf, inv);
    count_launch();
}

// x = M (f - mean f) on the coarsest level (FP64 arithmetic); without the
// mean when the operator has no null space (keep_mean).
template <typename T>
__global__ void coarse_solve_kernel(int n, const double* __restrict__ M, const T* __restrict__ f,
                                    T* __restrict__ x, int keep_mean) {
    extern __shared__ double fs[];
    __shared__ double mean;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int c = tid; c < n; c += nt) fs[c] = (double)f[c];
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int c = 0; c < n; ++c) t += fs[c];
        mean = keep_mean ? 0.0 : t / (double)n;
    }
    __syncthreads();
    for (int r = tid; r < n; r += nt) {
        double acc = 0.0;
        for (int c = 0; c < n; ++c) acc = fma(M[(int64_t)r * n + c], fs[c] - mean, acc);
        x[r] = (T)acc;
    }
}

template <typename T>
void launch_coarse_solve(const Geo& g, const double* inv, const T* f, T* x, cudaStream_t st, bool keep_mean) {
    int n = (int)g.ncell();
    coarse_solve_kernel<T><<<1, 128, sizeof(double) * n, st>>>(n, inv, f, x, keep_mean ? 1 : 0);
    count_launch();
}

// ------------------------------------------------------------------ smoothers ---

// Over-relaxed Gauss-Seidel update of Eq. eq:beta_pressure in the SPD form:
//   x_c <- x_c + omega ( w_c (f_c/scale + sum_f beta_f x_nb) - x_c ),
// w_c = 1/sum_f beta_f.  One thread per x-pair (2t, 2t+1) of a row updates
// the member of colour `color` ((i+j+k) even = red = 0).  With zero_init the
// incoming x is taken as zero and the other member of the pair is zeroed.

template <typename T, typename TB, bool USEW, bool I32>
__global__ void __launch_bounds__(kTX* pass_rows<T>()) rbgs_kernel(Geo g, const TB* __restrict__ bx,
                                                       const TB* __restrict__ by,
                                                       const TB* __restrict__ bz, T scale,
                                                       const T* __restrict__ w,
                                                       const T* __restrict__ f, T* __restrict__ x,
                                                       int color, T omega, int zero_init, int k0) {
    pdl_wait();
    const int t = blockIdx.x * kTX + threadIdx.x;
    const int j = blockIdx.y * pass_rows<T>() + threadIdx.y;
    const int k = k0 + blockIdx.z;
    const int i0 = 2 * t;
    if (i0 >= g.nx || j >= g.ny) return;
    const int i = i0 + ((i0 + j + k + color) & 1);
    const int io = i0 + 1 - (i - i0);  // the other member of the pair
    const T hs = T(1) / scale;
    if (i < g.nx) {
        Stencil<T> s;
        int64_t c;
        if (I32) {
            int c32;
            load_stencil_fast<T>(g, bx, by, bz, i, j, k, s, c32);
            c = c32;
        } else {
            c = g.cidx(i, j, k);
            load_stencil_as<T>(g, bx, by, bz, i, j, k, s);
        }
        T xn;
        if (zero_init) {
            const T wc = USEW ? w[c] : inv_sum6(s.b);
            xn = omega * wc * (f[c] * hs);
        } else {
            T acc = f[c] * hs;
#pragma unroll
            for (int q = 0; q < 6; ++q) acc = fma(s.b[q], x[s.nb[q]], acc);
            const T xc = x[c];
            xn = fma(omega, fma(USEW ? w[c] : inv_sum6(s.b), acc, -xc), xc);
        }
        x[c] = xn;
    }
    if (zero_init && io < g.nx) x[g.cidx(io, j, k)] = T(0);
}

// Four consecutive cells of a row as one 16-byte (FP32) or two 16-byte
// (FP64) loads.
template <typename T>
__device__ __forceinline__ void ld4(T (&d)[4], const T* __restrict__ p) {
    if constexpr (sizeof(T) == 4) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(p));
        d[0] = a.x; d[1] = a.y; d[2] = a.z; d[3] = a.w;
    } else {
        const double2 a = __ldg(reinterpret_cast<const double2*>(p));
        const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
        d[0] = a.x; d[1] = a.y; d[2] = b.x; d[3] = b.y;
    }
}
// four FP16 values widened to FP32 (one 8-byte load)
__device__ __forceinline__ void ld4(float (&d)[4], const __half* __restrict__ p) {
    const uint2 raw = __ldg(reinterpret_cast<const uint2*>(p));
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&raw.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&raw.y));
    d[0] = a.x;
    d[1] = a.y;
    d[2] = b.x;
    d[3] = b.y;
}
__device__ __forceinline__ float ldb(const float* __restrict__ p) { return __ldg(p); }
__device__ __forceinline__ double ldb(const double* __restrict__ p) { return __ldg(p); }
__device__ __forceinline__ float ldb(const __half* __restrict__ p) { return __half2float(__ldg(p)); }

template <typename T>
__device__ __forceinline__ void ld4x(T (&d)[4], const T* p) {  // x: written in the same pass
    if constexpr (sizeof(T) == 4) {
        const float4 a = *reinterpret_cast<const float4*>(p);
        d[0] = a.x; d[1] = a.y; d[2] = a.z; d[3] = a.w;
    } else {
        const double2 a = *reinterpret_cast<const double2*>(p);
        const double2 b = *(reinterpret_cast<const double2*>(p) + 1);
        d[0] = a.x; d[1] = a.y; d[2] = b.x; d[3] = b.y;
    }
}

// The colour pass of rbgs_kernel with two pairs per thread: cells 4q..4q+3
// of a row, of which the two of colour `color` are updated, every array read
// as 16-byte vectors (the single-pair kernel's scalar loads stream the level
// more slowly).  Same update, faces in the same order.  Needs nx % 4 == 0, no
// walls along x, 32-bit offsets and 16-byte aligned arrays.
// M: the updated member of both pairs ((j + k + color) & 1, uniform per warp).
// Returns the two new values (cells i0 + M and i0 + 2 + M); the caller stores.
template <typename T, typename TB, bool USEW, int M>
__device__ __forceinline__ void rbgs4_row(const Geo& g, const TB* __restrict__ bx, const TB* __restrict__ by,
                                          const TB* __restrict__ bz, T scale, const T* __restrict__ w,
                                          const T* __restrict__ f, const T* x, T omega, int zero_init,
                                          int j, int k, int i0, int lane, T (&out)[2]) {
    const int nx = g.nx, ny = g.ny, nz = g.nz, pl = nx * ny;
    const int rowc = (k * ny + j) * nx;
    const int c0 = rowc + i0;
    const bool ylo = j == 0, yhi = j == ny - 1, zlo = k == 0, zhi = k == nz - 1;
    const int ym = !ylo ? -nx : (g.wy ? 0 : (ny - 1) * nx), yp = !yhi ? nx : (g.wy ? 0 : -(ny - 1) * nx);
    const int zm = !zlo ? -pl : (g.wz ? 0 : (nz - 1) * pl), zp = !zhi ? pl : (g.wz ? 0 : -(nz - 1) * pl);
    const int fy0 = (k * (ny + g.wy) + j) * nx + i0;  // y-faces below the cells
    const int fy1 = (!yhi || g.wy) ? fy0 + nx : fy0 - (ny - 1) * nx;
    T X[4], F[4], W[4], XYM[4], XYP[4], XZM[4], XZP[4], BX[4], BY0[4], BY1[4], BZ0[4], BZ1[4];
    ld4(F, f + c0);
    if (USEW) ld4(W, w + c0);
    ld4(BX, bx + c0);  // x-faces i0 .. i0+3 (no walls along x: the face row is the cell row)
    ld4(BY0, by + fy0);
    ld4(BY1, by + fy1);
    ld4(BZ0, bz + c0);
    ld4(BZ1, bz + ((!zhi || g.wz) ? c0 + pl : c0 - (nz - 1) * pl));
    // face i0+4 (the + face of the last cell): the next lane's first, or loaded
    const int ir = i0 + 4 < nx ? i0 + 4 : 0;
    // (every lane takes part in the shuffle; the select comes after it)
    const T bxr_ld = (T)ldb(bx + rowc + ir);
    const T bxr_sh = __shfl_down_sync(0xffffffffu, BX[0], 1);
    const T bxr = (lane < kTX - 1 && i0 + 4 < nx) ? bxr_sh : bxr_ld;
    if (zero_init) {
#pragma unroll
        for (int u = 0; u < 4; ++u) X[u] = XYM[u] = XYP[u] = XZM[u] = XZP[u] = T(0);
    } else {
        ld4x(X, x + c0);
        ld4x(XYM, x + c0 + ym);
        ld4x(XYP, x + c0 + yp);
        ld4x(XZM, x + c0 + zm);
        ld4x(XZP, x + c0 + zp);
    }
    // x of the cells next to the quad (i0-1 and i0+4, wrapped around the row)
    T xl = T(0), xr = T(0);
    if (!zero_init) {
        const T xl_ld = x[rowc + (i0 > 0 ? i0 - 1 : nx - 1)], xr_ld = x[rowc + ir];
        const T xl_sh = __shfl_up_sync(0xffffffffu, X[3], 1), xr_sh = __shfl_down_sync(0xffffffffu, X[0], 1);
        xl = (lane > 0 && i0 > 0) ? xl_sh : xl_ld;
        xr = (lane < kTX - 1 && i0 + 4 < nx) ? xr_sh : xr_ld;
    }
    const T hs = T(1) / scale;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int li = 2 * u + M;  // the updated cell of pair u
        T b[6];
        b[0] = BX[li];
        b[1] = li < 3 ? BX[li + 1] : bxr;
        b[2] = (g.wy && ylo) ? T(0) : BY0[li];
        b[3] = (g.wy && yhi) ? T(0) : BY1[li];
        b[4] = (g.wz && zlo) ? T(0) : BZ0[li];
        b[5] = (g.wz && zhi) ? T(0) : BZ1[li];
        T xn;
        if (zero_init) {
            const T wc = USEW ? W[li] : inv_sum6(b);
            xn = omega * wc * (F[li] * hs);
        } else {
            const T nb[6] = {li > 0 ? X[li - 1] : xl, li < 3 ? X[li + 1] : xr, XYM[li], XYP[li], XZM[li], XZP[li]};
            T acc = F[li] * hs;
#pragma unroll
            for (int q = 0; q < 6; ++q) acc = fma(b[q], nb[q], acc);
            const T xc = X[li];
            xn = fma(omega, fma(USEW ? W[li] : inv_sum6(b), acc, -xc), xc);
        }
        out[u] = xn;
    }
}

// The row's two new values are computed before either is stored (the FP64
// form's passes measured 4 % faster so than with the stores inside the
// update).
template <typename T, bool USEW, typename TB = T>
__global__ void __launch_bounds__(kTX* pass_rows<T>()) rbgs4_kernel(Geo g, const TB* __restrict__ bx,
                                                        const TB* __restrict__ by,
                                                        const TB* __restrict__ bz, T scale,
                                                        const T* __restrict__ w,
                                                        const T* __restrict__ f, T* __restrict__ x,
                                                        int color, T omega, int zero_init, int k0) {
    pdl_wait();
    const int j = blockIdx.y * pass_rows<T>() + threadIdx.y;
    if (j >= g.ny) return;  // uniform per warp
    const int k = k0 + blockIdx.z;
    const int nq = g.nx / 4;
    const int lane = threadIdx.x;
    const int qv = blockIdx.x * kTX + lane;
    const bool act = qv < nq;
    const int i0 = 4 * (act ? qv : nq - 1);  // idle lanes shadow the last quad (no stores)
    const int M = (j + k + color) & 1;
    T xn[2];
    if (M == 0)
        rbgs4_row<T, TB, USEW, 0>(g, bx, by, bz, scale, w, f, x, omega, zero_init, j, k, i0, lane, xn);
    else
        rbgs4_row<T, TB, USEW, 1>(g, bx, by, bz, scale, w, f, x, omega, zero_init, j, k, i0, lane, xn);
    if (!act) return;
    const int c0 = (k * g.ny + j) * g.nx + i0;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int li = 2 * u + M;
        x[c0 + li] = xn[u];
        if (zero_init) x[c0 + li + 1 - 2 * M] = T(0);  // the other member of the pair
    }
}

template <typename T>
void launch_rbgs(const Geo& g, const Coef<T>& cf, const T* w, const T* f, T* x, int color,
                 double omega, bool zero_init, cudaStream_t st, int k0, int k1) {
    if (k1 < 0) k1 = g.nz;
    // four cells per thread where a row fills at least a warp (shorter rows
    // would leave lanes idle: the single-pair kernel serves them)
    if (g.nx % 4 == 0 && g.nx >= 4 * kTX && !g.wx && fits_i32(g) && aligned16(cf.bx, cf.by, cf.bz, f) &&
        aligned16(x) && ((sizeof(T) == 4 && !cf.sig) || aligned16(w))) {
        dim3 gr((g.nx / 4 + kTX - 1) / kTX, (g.ny + pass_rows<T>() - 1) / pass_rows<T>(), k1 - k0);
        if (sizeof(T) == 8 || cf.sig)  // w read (FP64, or a diagonal excess the coefficients do not hold)
            launch_pdl(rbgs4_kernel<T, true>, gr, dim3(kTX, pass_rows<T>()), 0, st, g, cf.bx, cf.by, cf.bz, cf.scale, w, f,
                x, color, (T)omega, zero_init ? 1 : 0, k0);
        else
            launch_pdl(rbgs4_kernel<T, false>, gr, dim3(kTX, pass_rows<T>()), 0, st, g, cf.bx, cf.by, cf.bz, cf.scale, w,
                f, x, color, (T)omega, zero_init ? 1 : 0, k0);
        count_launch();
        return;
    }
    const int npair = (g.nx + 1) / 2;
    dim3 gr((npair + kTX - 1) / kTX, (g.ny + pass_rows<T>() - 1) / pass_rows<T>(), k1 - k0);
    // FP32: recomputing 1/D from the coefficients already loaded is cheaper
    // than reading it; FP64: the division costs more than the read
    const bool i32 = fits_i32(g);
    if (sizeof(T) == 8 || cf.sig) {
        if (i32)
            launch_pdl(rbgs_kernel<T, T, true, true>, gr, dim3(kTX, pass_rows<T>()), 0, st, g, cf.bx, cf.by, cf.bz,
                cf.scale, w, f, x, color, (T)omega, zero_init ? 1 : 0, k0);
        else
            launch_pdl(rbgs_kernel<T, T, true, false>, gr, dim3(kTX, pass_rows<T>()), 0, st, g, cf.bx, cf.by, cf.bz,
                cf.scale, w, f, x, color, (T)omega, zero_init ? 1 : 0, k0);
    } else {
        if (i32)
            launch_pdl(rbgs_kernel<T, T, false, true>, gr, dim3(kTX, pass_rows<T>()), 0, st, g, cf.bx, cf.by, cf.bz,
                cf.scale, w, f, x, color, (T)omega, zero_init ? 1 : 0, k0);
        else
            launch_pdl(rbgs_kernel<T, T, false, false>, gr, dim3(kTX, pass_rows<T>()), 0, st, g, cf.bx, cf.by, cf.bz,
                cf.scale, w, f, x, color, (T)omega, zero_init ? 1 : 0, k0);
    }
    count_launch();
}

void launch_rbgs_h(const Geo& g, const __half* const b[3], float scale, const float* f, float* x,
                   int color, double omega, bool zero_init, cudaStream_t st, int k0, int k1) {
    if (k1 < 0) k1 = g.nz;
    // four cells per thread where a row fills a warp (the update of the pair kernel)
    if (g.nx % 4 == 0 && g.nx >= 4 * kTX && !g.wx && fits_i32(g) && aligned16(f, x) &&
        ((((uintptr_t)b[0] | (uintptr_t)b[1] | (uintptr_t)b[2]) & 7u) == 0)) {
        dim3 gr((g.nx / 4 + kTX - 1) / kTX, (g.ny + pass_rows<float>() - 1) / pass_rows<float>(), k1 - k0);
        launch_pdl(rbgs4_kernel<float, false, __half>, gr, dim3(kTX, pass_rows<float>()), 0, st, g, b[0], b[1], b[2], scale,
                   (const float*)nullptr, f, x, color, (float)omega, zero_init ? 1 : 0, k0);
        count_launch();
        return;
    }
    const int npair = (g.nx + 1) / 2;
    dim3 gr((npair + kTX - 1) / kTX, (g.ny + pass_rows<float>() - 1) / pass_rows<float>(), k1 - k0);
    if (fits_i32(g))
        launch_pdl(rbgs_kernel<float, __half, false, true>, gr, dim3(kTX, pass_rows<float>()), 0, st, g, b[0], b[1], b[2],
            scale, nullptr, f, x, color, (float)omega, zero_init ? 1 : 0, k0);
    else
        launch_pdl(rbgs_kernel<float, __half, false, false>, gr, dim3(kTX, pass_rows<float>()), 0, st, g, b[0], b[1], b[2],
            scale, nullptr, f, x, color, (float)omega, zero_init ? 1 : 0, k0);
    count_launch();
}

// Damped Jacobi (the paper's GPU iteration, Sec. 3.7.4), double-buffered:
//   x_out = x + omega (w (f/scale + sum beta x_nb) - x).
template <typename T>
__global__ void __launch_bounds__(kTX* kTY) jacobi_kernel(Geo g, Coef<T> cf,
                                                         const T* __restrict__ w,
                                                         const T* __restrict__ f,
                                                         const T* __restrict__ x,
                                                         T* __restrict__ xo, T omega,
                                                         int zero_init) {
    const int i = blockIdx.x * kTX + threadIdx.x;
    const int j = blockIdx.y * kTY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const int64_t c = g.cidx(i, j, k);
    const T hs = T(1) / cf.scale;
    if (zero_init) {
        xo[c] = omega * w[c] * (f[c] * hs);
        return;
    }
    Stencil<T> s;
    load_stencil(g, cf, i, j, k, s);
    T acc = f[c] * hs;
#pragma unroll
    for (int q = 0; q < 6; ++q) acc = fma(s.b[q], x[s.nb[q]], acc);
    const T xc = x[c];
    xo[c] = fma(omega, fma(w[c], acc, -xc), xc);
}

template <typename T>
void launch_jacobi(const Geo& g, const Coef<T>& cf, const T* w, const T* f, const T* x, T* xout,
                   double omega, bool zero_init, cudaStream_t st) {
    dim3 gr((g.nx + kTX - 1) / kTX, (g.ny + kTY - 1) / kTY, g.nz);
    jacobi_kernel<T><<<gr, dim3(kTX, kTY), 0, st>>>(g, cf, w, f, x, xout, (T)omega,
                                                    zero_init ? 1 : 0);
    count_launch();
}

// ------------------------------------------------- restriction / prolongation ---

// Coarse right-hand side: the average over the children of the fine residual
// f - A x (restriction R = P^T / #children for the piecewise-constant P),
// each child's A x on its faces on the coarse cell's surface only (the
// faces between children cancel in the sum; apply_A_faces).  FULL: the
// 2 x 2 x 2 children of full coarsening, the loops unrolled so that the
// loads of all eight children are in flight together (the sum keeps its
// order).
template <typename T, typename TB, bool I32, bool SIG = false, bool FULL = false>
__global__ void restrict_residual_kernel(Geo fg, const TB* __restrict__ bx, const TB* __restrict__ by,
                                         const TB* __restrict__ bz, T scale, const T* __restrict__ f,
                                         const T* __restrict__ x, Geo cg, int fa0, int fa1,
                                         int fa2, T* __restrict__ fc, const T* __restrict__ sig) {
    pdl_wait();
    const int I = blockIdx.x * kTX + threadIdx.x;
    const int J = blockIdx.y * kTY + threadIdx.y;
    const int K = blockIdx.z;
    if (I >= cg.nx || J >= cg.ny) return;
    if (FULL) fa0 = fa1 = fa2 = 2;
    T sum = T(0);
#pragma unroll
    for (int dk = 0; dk < (FULL ? 2 : fa2); ++dk)
#pragma unroll
        for (int dj = 0; dj < (FULL ? 2 : fa1); ++dj)
#pragma unroll
            for (int di = 0; di < (FULL ? 2 : fa0); ++di) {
                const int i = I * fa0 + di, j = J * fa1 + dj, k = K * fa2 + dk;
                Stencil<T> s;
                int64_t c;
                if (I32) {
                    int c32;
                    load_stencil_fast<T>(fg, bx, by, bz, i, j, k, s, c32);
                    c = c32;
                } else {
                    c = fg.cidx(i, j, k);
                    load_stencil_as<T>(fg, bx, by, bz, i, j, k, s);
                }
                T ax = apply_A_faces(s, x, x[c], scale, surface_faces(di, dj, dk, fa0, fa1, fa2));
                if (SIG) ax = fma(scale * sig[c], x[c], ax);
                sum += f[c] - ax;
            }
    fc[cg.cidx(I, J, K)] = sum / T(fa0 * fa1 * fa2);
}

template <typename T>
void launch_restrict_residual(const Geo& fine, const Coef<T>& cf, const T* f, const T* x,
                             const Geo& coarse, const int fac[3], T* fc, cudaStream_t st) {
    dim3 gr((coarse.nx + kTX - 1) / kTX, (coarse.ny + kTY - 1) / kTY, coarse.nz);
    // the diagonal excess as a template flag: the plain operator's kernels are unchanged
    const bool full = fac[0] == 2 && fac[1] == 2 && fac[2] == 2;
    auto* k = fits_i32(fine)
                  ? (cf.sig ? restrict_residual_kernel<T, T, true, true>
                            : (full ? restrict_residual_kernel<T, T, true, false, true> : restrict_residual_kernel<T, T, true>))
                  : (cf.sig ? restrict_residual_kernel<T, T, false, true> : restrict_residual_kernel<T, T, false>);
    launch_pdl(k, gr, dim3(kTX, kTY), 0, st, fine, cf.bx, cf.by, cf.bz, cf.scale, f, x, coarse, fac[0], fac[1],
               fac[2], fc, cf.sig);
    count_launch();
}

void launch_restrict_residual_h(const Geo& fine, const __half* const b[3], float scale, const float* f,
                                const float* x, const Geo& coarse, const int fac[3], float* fc,
                                cudaStream_t st) {
    dim3 gr((coarse.nx + kTX - 1) / kTX, (coarse.ny + kTY - 1) / kTY, coarse.nz);
    if (fits_i32(fine) && fac[0] == 2 && fac[1] == 2 && fac[2] == 2)
        launch_pdl(restrict_residual_kernel<float, __half, true, false, true>, gr, dim3(kTX, kTY), 0, st, fine,
                   b[0], b[1], b[2], scale, f, x, coarse, fac[0], fac[1], fac[2], fc, (const float*)nullptr);
    else if (fits_i32(fine))
        launch_pdl(restrict_residual_kernel<float, __half, true>, gr, dim3(kTX, kTY), 0, st, fine, b[0], b[1],
            b[2], scale, f, x, coarse, fac[0], fac[1], fac[2], fc, (const float*)nullptr);
    else
        launch_pdl(restrict_residual_kernel<float, __half, false>, gr, dim3(kTX, kTY), 0, st, fine, b[0], b[1],
            b[2], scale, f, x, coarse, fac[0], fac[1], fac[2], fc, (const float*)nullptr);
    count_launch();
}

// FP16 copies of the (unscaled) face coefficients for the level-0 V-cycle
__global__ void convert_beta_half_kernel(int64_t n, const double* __restrict__ b, __half* __restrict__ out) {
    PARIS_EW_FOR(c, n) out[c] = __double2half(b[c]);
}

void launch_convert_beta_half(const Geo& g, const double* const b64[3], __half* const out[3],
                              cudaStream_t st) {
    for (int a = 0; a < 3; ++a) {
        const int64_t n = g.nface(a);
        convert_beta_half_kernel<<<elementwise_blocks(n), kRedThreads, 0, st>>>(n, b64[a], out[a]);
        count_launch();
    }
}

template <typename T>
__global__ void prolong_add_kernel(Geo fg, Geo cg, int fa0, int fa1, int fa2,
                                   const T* __restrict__ xc, T* __restrict__ x) {
    pdl_wait();
    const int i = blockIdx.x * kTX + threadIdx.x;
    const int j = blockIdx.y * kTY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= fg.nx || j >= fg.ny) return;
    // factors are 1 or 2: halving is a shift
    x[fg.cidx(i, j, k)] += xc[cg.cidx(i >> (fa0 - 1), j >> (fa1 - 1), k >> (fa2 - 1))];
}

// x_fine += x_coarse[parent] for four x-consecutive fine cells per thread
// (all axes halved, nx % 4 == 0, 16-byte aligned x)
__global__ void prolong_add4_kernel(Geo fg, Geo cg, const float* __restrict__ xc, float* __restrict__ x) {
    pdl_wait();
    const int q = blockIdx.x * kTX + threadIdx.x;  // quad index along x
    const int j = blockIdx.y * kTY + threadIdx.y;
    const int k = blockIdx.z;
    if (4 * q >= fg.nx || j >= fg.ny) return;
    const int64_t c = fg.cidx(4 * q, j, k);
    const int64_t cc = cg.cidx(2 * q, j >> 1, k >> 1);
    float4 v = *reinterpret_cast<const float4*>(x + c);
    const float a = xc[cc], b = xc[cc + 1];
    v.x += a;
    v.y += a;
    v.z += b;
    v.w += b;
    *reinterpret_cast<float4*>(x + c) = v;
}

template <typename T>
void launch_prolong_add(const Geo& fine, const Geo& coarse, const int fac[3], const T* xc, T* x,
                        cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        if (fac[0] == 2 && fac[1] == 2 && fac[2] == 2 && fine.nx % 4 == 0 && aligned16(x)) {
            dim3 gr((fine.nx / 4 + kTX - 1) / kTX, (fine.ny + kTY - 1) / kTY, fine.nz);
            launch_pdl(prolong_add4_kernel, gr, dim3(kTX, kTY), 0, st, fine, coarse, (const float*)xc,
                (float*)x);
            count_launch();
            return;
        }
    }
    dim3 gr((fine.nx + kTX - 1) / kTX, (fine.ny + kTY - 1) / kTY, fine.nz);
    launch_pdl(prolong_add_kernel<T>, gr, dim3(kTX, kTY), 0, st, fine, coarse, fac[0], fac[1], fac[2], xc, x);
    count_launch();
}

// ------------------------------------------------------------------ Krylov ---

// FP64 residual r = f - A x with fused norms; the mixed form also writes the
// scaled FP32 copy r32 = scale * r that the inner solve starts from.  With
// zero_ok and an initial guess that is zero everywhere (s->xmax == 0, a value
// every thread reads alike) A x vanishes and r = f is copied.
template <bool I32, bool SIG = false>
__global__ void __launch_bounds__(kTX* kTY) residual64_kernel(Geo g, Coef<double> cf,
                                                              const double* __restrict__ f,
                                                              const double* __restrict__ x,
                                                              double* __restrict__ r64,
                                                              float* __restrict__ r32,
                                                              const Scal* s, double* partials,
                                                              int zero_ok, int split, FinSpec fin) {
    pdl_wait();
    const int i = blockIdx.x * kTX + threadIdx.x;
    const int j = blockIdx.y * kTY + threadIdx.y;
    double l2 = 0.0;
    unsigned long long rmax_k = 0;
    unsigned nf = 0;
    if (i < g.nx && j < g.ny) {
        const int se = r32 ? (int)s->scale_exp : 0;
        const bool zero = zero_ok && s->xmax == 0.0;
        const int k0 = blockIdx.z * kZ, k1 = min(k0 + kZ, g.nz);
        PARIS_ZLOOP(k0, k1, {
            int64_t c;
            double r;
            if (zero) {
                c = g.cidx(i, j, k);
                r = f[c];
            } else {
                Stencil<double> st;
                if (I32) {
                    int c32;
                    load_stencil_fast<double>(g, cf.bx, cf.by, cf.bz, i, j, k, st, c32);
                    c = c32;
                } else {
                    c = g.cidx(i, j, k);
                    load_stencil(g, cf, i, j, k, st);
                }
                // (A x)/scale in the difference form, then one fused step
                const double xc = x[c];
                double a = st.b[0] * (xc - x[st.nb[0]]);
#pragma unroll
                for (int q = 1; q < 6; ++q) a = fma(st.b[q], xc - x[st.nb[q]], a);
                if (SIG) a = fma(cf.sig[c], xc, a);
                r = fma(-cf.scale, a, f[c]);
            }
            if (r64) r64[c] = r;
            if (r32) {
                // split: r32 in the colour-split layout (cell i of a row at
                // i/2, plus nx/2 for colour (i+j+k) odd)
                const int64_t cs = split ? c - i + (((i + j + k) & 1) ? g.nx / 2 : 0) + (i >> 1) : c;
                r32[cs] = d2f_scaled(r, se);
            }
            l2 = fma(r, r, l2);
            const unsigned long long kr = abs_key(r);
            rmax_k = kr > rmax_k ? kr : rmax_k;
            nf += key_nonfinite(kr);
        })
    }
    block_reduce_skc<double>(l2, rmax_k, nf, partials, flat_block(), flat_tid());
    finalize_last_block(partials, (int64_t)gridDim.x * gridDim.y * gridDim.z, fin, flat_tid());
}

int64_t launch_residual64(const Geo& g, const Coef<double>& cf, const double* f, const double* x,
                          double* r64, float* r32, const Scal* s, double* partials, bool zero_ok,
                          cudaStream_t st, FinSpec fin, bool split) {
    dim3 gr = tile_grid(g, kZ);
    auto* k = fits_i32(g) ? (cf.sig ? residual64_kernel<true, true> : residual64_kernel<true>)
                          : (cf.sig ? residual64_kernel<false, true> : residual64_kernel<false>);
    launch_pdl(k, gr, dim3(kTX, kTY), 0, st, g, cf, f, x, r64, r32, s, partials, zero_ok ? 1 : 0, split ? 1 : 0,
               fin);
    count_launch();
    return nblocks_of(gr);
}

// q = A d and the partial sums of d . q (accumulated per thread in T,
// across threads and blocks in FP64).
template <typename T, bool I32, bool SIG = false>
__global__ void __launch_bounds__(kTX* kTY) matvec_dot_kernel(Geo g, Coef<T> cf,
                                                             const T* __restrict__ d,
                                                             T* __restrict__ q,
                                                             double* partials, FinSpec fin) {
    const int i = blockIdx.x * kTX + threadIdx.x;
    const int j = blockIdx.y * kTY + threadIdx.y;
    T loc = T(0);
    if (i < g.nx && j < g.ny) {
        const int k0 = blockIdx.z * kZ, k1 = min(k0 + kZ, g.nz);
        PARIS_ZLOOP(k0, k1, {
            Stencil<T> st;
            int64_t c;
            if (I32) {
                int c32;
                load_stencil_fast<T>(g, cf.bx, cf.by, cf.bz, i, j, k, st, c32);
                c = c32;
            } else {
                c = g.cidx(i, j, k);
                load_stencil(g, cf, i, j, k, st);
            }
            const T dc = d[c];
            T qc = apply_A(st, d, dc, cf.scale);
            if (SIG) qc = fma(cf.scale * cf.sig[c], dc, qc);
            q[c] = qc;
            loc = fma(dc, qc, loc);
        })
    }
    double acc[1] = {(double)loc};
    const int op[1] = {0};
    block_reduce_store<1>(acc, op, partials, flat_block(), flat_tid());
    finalize_last_block(partials, (int64_t)gridDim.x * gridDim.y * gridDim.z, fin, flat_tid());
}

template <typename T>
int64_t launch_matvec_dot(const Geo& g, const Coef<T>& cf, const T* d, T* q, double* partials,
                          cudaStream_t st, FinSpec fin) {
    dim3 gr = tile_grid(g, kZ);
    auto* k = fits_i32(g) ? (cf.sig ? matvec_dot_kernel<T, true, true> : matvec_dot_kernel<T, true>)
                          : (cf.sig ? matvec_dot_kernel<T, false, true> : matvec_dot_kernel<T, false>);
    k<<<gr, dim3(kTX, kTY), 0, st>>>(g, cf, d, q, partials, fin);
    count_launch();
    return nblocks_of(gr);
}

// The streaming Krylov kernels keep several independent 16-byte loads per
// array in flight per thread (kKU iterations of the grid-stride loop at once,
// each with its own partial sums), which the memory system needs to stream
// at its rate; the partial sums are folded in a fixed order.
#ifndef PARIS_KU
#define PARIS_KU 4
#endif
constexpr int kKU = PARIS_KU;

// NOX: r only (d and x not touched), the same loops and partial sums
template <typename T, bool NOX = false>
__global__ void update_xr_kernel(int64_t n, const Scal* s, const T* __restrict__ d,
                                 const T* __restrict__ q, T* __restrict__ x, T* __restrict__ r,
                                 double* partials, int vec, FinSpec fin, int rev) {
    using VT = typename V16<T>::type;
    constexpr int W = V16<T>::n;
    constexpr int U = kKU / 2;  // four arrays per element: two iterations at once
    pdl_wait();
    const T alpha = (T)s->alpha;
    T l2[U], li[U];
#pragma unroll
    for (int u = 0; u < U; ++u) l2[u] = li[u] = T(0);
    unsigned nf = 0;  // an integer count: no FP64 add per element
    auto one = [&](T dv, T qv, T& xv, T& rv, T& l2u, T& liu) {
        if (!NOX) xv = fma(alpha, dv, xv);
        rv = fma(-alpha, qv, rv);
        l2u = fma(rv, rv, l2u);
        liu = fmax(liu, fabs(rv));
        nf += isfinite(rv) ? 0u : 1u;
    };
    const int64_t nv = vec ? n / W : 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // rev: the vectors from the end (a pass that starts where the previous one ended)
    auto at = [&](int64_t e) { return rev ? nv - 1 - e : e; };
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + (U - 1) * stride < nv; i += U * stride) {
        VT dv[U], qv[U], xv[U], rv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!NOX) dv[u] = reinterpret_cast<const VT*>(d)[at(i + u * stride)];
            qv[u] = reinterpret_cast<const VT*>(q)[at(i + u * stride)];
            if (!NOX) xv[u] = reinterpret_cast<VT*>(x)[at(i + u * stride)];
            rv[u] = reinterpret_cast<VT*>(r)[at(i + u * stride)];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const T* de = reinterpret_cast<const T*>(&dv[u]);
            const T* qe = reinterpret_cast<const T*>(&qv[u]);
            T* xe = reinterpret_cast<T*>(&xv[u]);
            T* re = reinterpret_cast<T*>(&rv[u]);
#pragma unroll
            for (int w = 0; w < W; ++w) one(de[w], qe[w], xe[w], re[w], l2[u], li[u]);
            if (!NOX) reinterpret_cast<VT*>(x)[at(i + u * stride)] = xv[u];
            reinterpret_cast<VT*>(r)[at(i + u * stride)] = rv[u];
        }
    }
    for (; i < nv; i += stride) {
        VT dv, xv;
        if (!NOX) {
            dv = reinterpret_cast<const VT*>(d)[at(i)];
            xv = reinterpret_cast<VT*>(x)[at(i)];
        }
        const VT qv = reinterpret_cast<const VT*>(q)[at(i)];
        VT rv = reinterpret_cast<VT*>(r)[at(i)];
        const T* de = reinterpret_cast<const T*>(&dv);
        const T* qe = reinterpret_cast<const T*>(&qv);
        T* xe = reinterpret_cast<T*>(&xv);
        T* re = reinterpret_cast<T*>(&rv);
#pragma unroll
        for (int w = 0; w < W; ++w) one(de[w], qe[w], xe[w], re[w], l2[0], li[0]);
        if (!NOX) reinterpret_cast<VT*>(x)[at(i)] = xv;
        reinterpret_cast<VT*>(r)[at(i)] = rv;
    }
    PARIS_TAIL_FOR(c, nv * W, n) {
        T xv = NOX ? T(0) : x[c], rv = r[c];
        one(NOX ? T(0) : d[c], q[c], xv, rv, l2[0], li[0]);
        if (!NOX) x[c] = xv;
        r[c] = rv;
    }
    T l2s = l2[0], lis = li[0];
#pragma unroll
    for (int u = 1; u < U; ++u) {
        l2s += l2[u];
        lis = fmax(lis, li[u]);
    }
    double acc[3] = {(double)l2s, (double)lis, (double)nf};
    const int op[3] = {0, 1, 0};
    block_reduce_store<3>(acc, op, partials, blockIdx.x, threadIdx.x);
    finalize_last_block(partials, gridDim.x, fin, threadIdx.x);
}

template <typename T>
int64_t launch_update_xr(int64_t n, const Scal* s, const T* d, const T* q, T* x, T* r,
                         double* partials, cudaStream_t st, FinSpec fin, bool rev) {
    int nb = elementwise_blocks(n);
    launch_pdl(update_xr_kernel<T>, dim3(nb), dim3(kRedThreads), 0, st, n, s, d, q, x, r, partials,
               aligned16(d, q, x, r) ? 1 : 0, fin, rev ? 1 : 0);
    count_launch();
    return nb;
}

template <typename T>
int64_t launch_update_r(int64_t n, const Scal* s, const T* q, T* r, double* partials, cudaStream_t st, FinSpec fin,
                        bool rev) {
    int nb = elementwise_blocks(n);
    launch_pdl(update_xr_kernel<T, true>, dim3(nb), dim3(kRedThreads), 0, st, n, s, (const T*)nullptr, q, (T*)nullptr,
               r, partials, aligned16(q, r) ? 1 : 0, fin, rev ? 1 : 0);
    count_launch();
    return nb;
}

template <typename T>
__global__ void dot2_kernel(int64_t n, const T* __restrict__ a, const T* __restrict__ b,
                            const T* __restrict__ c, double* partials, int vec, FinSpec fin, int rev) {
    using VT = typename V16<T>::type;
    constexpr int W = V16<T>::n;
    constexpr int U = kKU;
    pdl_wait();
    T s0[U], s1[U];
#pragma unroll
    for (int u = 0; u < U; ++u) s0[u] = s1[u] = T(0);
    const int64_t nv = vec ? n / W : 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    auto at = [&](int64_t e) { return rev ? nv - 1 - e : e; };  // rev: from the end
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + (U - 1) * stride < nv; i += U * stride) {
        VT av[U], bv[U], cv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            av[u] = __ldg(reinterpret_cast<const VT*>(a) + at(i + u * stride));
            bv[u] = __ldg(reinterpret_cast<const VT*>(b) + at(i + u * stride));
            if (c) cv[u] = __ldg(reinterpret_cast<const VT*>(c) + at(i + u * stride));
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const T* ae = reinterpret_cast<const T*>(&av[u]);
            const T* be = reinterpret_cast<const T*>(&bv[u]);
#pragma unroll
            for (int w = 0; w < W; ++w) s0[u] = fma(ae[w], be[w], s0[u]);
            if (c) {
                const T* ce = reinterpret_cast<const T*>(&cv[u]);
#pragma unroll
                for (int w = 0; w < W; ++w) s1[u] = fma(ae[w], ce[w], s1[u]);
            }
        }
    }
    for (; i < nv; i += stride) {
        const VT av = reinterpret_cast<const VT*>(a)[at(i)];
        const VT bv = reinterpret_cast<const VT*>(b)[at(i)];
        const T* ae = reinterpret_cast<const T*>(&av);
        const T* be = reinterpret_cast<const T*>(&bv);
#pragma unroll
        for (int w = 0; w < W; ++w) s0[0] = fma(ae[w], be[w], s0[0]);
        if (c) {
            const VT cv = reinterpret_cast<const VT*>(c)[at(i)];
            const T* ce = reinterpret_cast<const T*>(&cv);
#pragma unroll
            for (int w = 0; w < W; ++w) s1[0] = fma(ae[w], ce[w], s1[0]);
        }
    }
    PARIS_TAIL_FOR(e, nv * W, n) {
        s0[0] = fma(a[e], b[e], s0[0]);
        if (c) s1[0] = fma(a[e], c[e], s1[0]);
    }
    T t0, t1;
    if constexpr (U == 4) {
        t0 = (s0[0] + s0[1]) + (s0[2] + s0[3]);
        t1 = (s1[0] + s1[1]) + (s1[2] + s1[3]);
    } else {
        t0 = s0[0];
        t1 = s1[0];
#pragma unroll
        for (int u = 1; u < U; ++u) {
            t0 += s0[u];
            t1 += s1[u];
        }
    }
    double acc[2] = {(double)t0, (double)t1};
    const int op[2] = {0, 0};
    block_reduce_store<2>(acc, op, partials, blockIdx.x, threadIdx.x);
    finalize_last_block(partials, gridDim.x, fin, threadIdx.x);
}

template <typename T>
int64_t launch_dot2(int64_t n, const T* a, const T* b, const T* c, double* partials,
                    cudaStream_t st, FinSpec fin, bool rev) {
    int nb = elementwise_blocks(n);
    launch_pdl(dot2_kernel<T>, dim3(nb), dim3(kRedThreads), 0, st, n, a, b, c, partials,
               aligned16(a, b, c) ? 1 : 0, fin, rev ? 1 : 0);
    count_launch();
    return nb;
}

template <typename T>
__global__ void xpby_kernel(int64_t n, const Scal* s, const T* __restrict__ z, T* __restrict__ d,
                            int vec) {
    using VT = typename V16<T>::type;
    constexpr int W = V16<T>::n;
    pdl_wait();
    const T beta = (T)s->beta;
    const int64_t nv = vec ? n / W : 0;
    PARIS_VEC_FOR(i, nv) {
        const VT zv = reinterpret_cast<const VT*>(z)[i];
        VT dv = reinterpret_cast<VT*>(d)[i];
        const T* ze = reinterpret_cast<const T*>(&zv);
        T* de = reinterpret_cast<T*>(&dv);
#pragma unroll
        for (int w = 0; w < W; ++w) de[w] = fma(beta, de[w], ze[w]);
        reinterpret_cast<VT*>(d)[i] = dv;
    }
    PARIS_TAIL_FOR(e, nv * W, n) d[e] = fma(beta, d[e], z[e]);
}

template <typename T>
void launch_xpby(int64_t n, const Scal* s, const T* z, T* d, cudaStream_t st) {
    launch_pdl(xpby_kernel<T>, dim3(elementwise_blocks(n)), dim3(kRedThreads), 0, st, n, s, z, d,
               aligned16(z, d) ? 1 : 0);
    count_launch();
}

// x += e * inv_scale, inv_scale a power of two: the product is the exact
// conversion with an exponent shift, then one FP64 addition.
__global__ void accumulate_kernel(int64_t n, const Scal* s, const float* __restrict__ e,
                                  double* __restrict__ x, int vec) {
    pdl_wait();
    const int sh = -(int)s->scale_exp;
    const int64_t nv = vec ? n / 4 : 0;
    PARIS_VEC_FOR(i, nv) {
        const float4 ev = reinterpret_cast<const float4*>(e)[i];
        double2 x0 = reinterpret_cast<double2*>(x)[2 * i];
        double2 x1 = reinterpret_cast<double2*>(x)[2 * i + 1];
        x0.x += f2d_scaled(ev.x, sh);
        x0.y += f2d_scaled(ev.y, sh);
        x1.x += f2d_scaled(ev.z, sh);
        x1.y += f2d_scaled(ev.w, sh);
        reinterpret_cast<double2*>(x)[2 * i] = x0;
        reinterpret_cast<double2*>(x)[2 * i + 1] = x1;
    }
    PARIS_TAIL_FOR(c, nv * 4, n) x[c] += f2d_scaled(e[c], sh);
}

void launch_accumulate(int64_t n, const Scal* s, const float* e, double* x, cudaStream_t st) {
    launch_pdl(accumulate_kernel, elementwise_blocks(n), kRedThreads, 0, st, n, s, e, x,
               aligned16(e, x) ? 1 : 0);
    count_launch();
}

// ------------------------------------------------------------- self-check ---

__global__ void check_arithmetic_kernel(const double* __restrict__ v, int64_t n, int shift, double p2,
                                        unsigned long long* bad) {
    unsigned long long cnt = 0;
    PARIS_EW_FOR(i, n) {
        const double x = v[i];
        // FP64 -> FP32 with the scaling 2^shift (the product by p2 = 2^shift is exact)
        const float hw = __double2float_rn(x * p2);
        const float sw = d2f_scaled(x, shift);
        const bool hw_sub = hw != 0.0f && fabsf(hw) < 1.17549435e-38f;  // flushed by design
        if (isnan(hw)) cnt += isnan(sw) ? 0 : 1;
        else if (hw_sub) cnt += (sw == 0.0f) ? 0 : 1;
        else cnt += (__float_as_int(hw) == __float_as_int(sw)) ? 0 : 1;
        // FP32 -> FP64 with 2^-shift (exact in both)
        if (!isnan(hw) && !hw_sub) {
            const double hw2 = (double)hw / p2;
            const double sw2 = f2d_scaled(hw, -shift);
            cnt += (__double_as_longlong(hw2) == __double_as_longlong(sw2)) ? 0 : 1;
        }
        // reciprocal within one ulp of the correctly rounded quotient
        if (x > 0.0 && x >= 0x1p-123 && x < 0x1p117) {
            const long long a = __double_as_longlong(recip64(x)), b = __double_as_longlong(1.0 / x);
            cnt += (a - b <= 1 && b - a <= 1) ? 0 : 1;
        }
    }
    if (cnt) atomicAdd(bad, cnt);
}

void launch_check_arithmetic(const double* v, int64_t n, int shift, unsigned long long* bad,
                             cudaStream_t st) {
    check_arithmetic_kernel<<<elementwise_blocks(n), kRedThreads, 0, st>>>(v, n, shift, ldexp(1.0, shift), bad);
    count_launch();
}

// --------------------------------------------------- streaming probes ---

// Reads a, b and c once: the rate of a read-only stream.  Each thread keeps
// kReadUnroll independent 16-byte loads of every array in flight (12 loads
// per iteration), so the grid holds enough bytes in flight to cover the
// memory latency; the sum a.(b + c) per warp goes to o[warp] so that the
// loads stay live.
constexpr int kReadUnroll = 4;
__global__ void __launch_bounds__(kRedThreads) stream_read3_kernel(const float4* __restrict__ a,
                                                                   const float4* __restrict__ b,
                                                                   const float4* __restrict__ c,
                                                                   float* __restrict__ o, int64_t nv) {
    float s = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + (kReadUnroll - 1) * stride < nv; i += kReadUnroll * stride) {
        float4 x[kReadUnroll], y[kReadUnroll], z[kReadUnroll];
#pragma unroll
        for (int u = 0; u < kReadUnroll; ++u) {
            x[u] = __ldcs(a + i + u * stride);
            y[u] = __ldcs(b + i + u * stride);
            z[u] = __ldcs(c + i + u * stride);
        }
#pragma unroll
        for (int u = 0; u < kReadUnroll; ++u) {
            s = fmaf(x[u].x, y[u].x + z[u].x, s);
            s = fmaf(x[u].y, y[u].y + z[u].y, s);
            s = fmaf(x[u].z, y[u].z + z[u].z, s);
            s = fmaf(x[u].w, y[u].w + z[u].w, s);
        }
    }
    for (; i < nv; i += stride) {
        const float4 x = __ldcs(a + i), y = __ldcs(b + i), z = __ldcs(c + i);
        s = fmaf(x.x, y.x + z.x, s);
        s = fmaf(x.y, y.y + z.y, s);
        s = fmaf(x.z, y.z + z.z, s);
        s = fmaf(x.w, y.w + z.w, s);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if ((threadIdx.x & 31) == 0) o[((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5] = s;
}

// o = a + 0.5 b: two streams read, one written
__global__ void stream_triad_kernel(const float4* __restrict__ a, const float4* __restrict__ b,
                                    float4* __restrict__ o, int64_t nv) {
    PARIS_VEC_FOR(i, nv) {
        const float4 x = a[i], y = b[i];
        o[i] = make_float4(fmaf(0.5f, y.x, x.x), fmaf(0.5f, y.y, x.y), fmaf(0.5f, y.z, x.z), fmaf(0.5f, y.w, x.w));
    }
}

cudaError_t stream_rates(const float* a, const float* b, const float* c, float* o, int64_t n, int reps,
                         double* read_gbs, double* triad_gbs, cudaStream_t st) {
    const int64_t nv = n / 4;
    // every SM full of resident blocks, one wave (the loops stride over the rest)
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stream_read3_kernel, kRedThreads, 0) !=
            cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    // o receives one float per warp of the read kernel: at most n/4 of them
    const int64_t cap = std::max<int64_t>(1, nv * 32 / kRedThreads);
    const int nb = (int)std::min<int64_t>((int64_t)device_sms() * per_sm, cap);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best_r = 1e30f, best_t = 1e30f;
    for (int r = 0; e == cudaSuccess && r <= reps; ++r) {
        float ms = 0.f;
        cudaEventRecord(e0, st);
        stream_read3_kernel<<<nb, kRedThreads, 0, st>>>((const float4*)a, (const float4*)b, (const float4*)c, o, nv);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && ms < best_r) best_r = ms;  // the first run warms up
        cudaEventRecord(e0, st);
        stream_triad_kernel<<<nb, kRedThreads, 0, st>>>((const float4*)a, (const float4*)b, (float4*)o, nv);
        cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && ms < best_t) best_t = ms;
        count_launch(2);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    *read_gbs = 3.0 * 16.0 * nv / (best_r * 1e-3) / 1e9;
    *triad_gbs = 3.0 * 16.0 * nv / (best_t * 1e-3) / 1e9;
    return e;
}

// ------------------------------------------------------ explicit instances ---

#define PARIS_INSTANTIATE(T)                                                                  \
    template void launch_convert_beta<T>(const Geo&, const double* [3], double, T* [3],        \
                                         cudaStream_t);                                        \
    template void launch_coarse_beta<T>(const Geo&, const Coef<T>&, const Geo&, const int[3],  \
                                        const double[3], T* [3], cudaStream_t);                \
    template void launch_inv_diag<T>(const Geo&, const Coef<T>&, T*, cudaStream_t);            \
    template void launch_coarse_inverse<T>(const Geo&, const Coef<T>&, double*, cudaStream_t); \
    template void launch_coarse_solve<T>(const Geo&, const double*, const T*, T*, cudaStream_t, bool); \
    template void launch_coarse_sig<T>(const Geo&, const T*, double, const Geo&, const int[3], T*,     \
                                       cudaStream_t);                                                  \
    template void launch_rbgs<T>(const Geo&, const Coef<T>&, const T*, const T*, T*, int,     \
                                 double, bool, cudaStream_t, int, int);                        \
    template void launch_jacobi<T>(const Geo&, const Coef<T>&, const T*, const T*, const T*,  \
                                   T*, double, bool, cudaStream_t);                            \
    template void launch_restrict_residual<T>(const Geo&, const Coef<T>&, const T*, const T*,  \
                                              const Geo&, const int[3], T*, cudaStream_t);     \
    template void launch_prolong_add<T>(const Geo&, const Geo&, const int[3], const T*, T*,   \
                                        cudaStream_t);                                         \
    template int64_t launch_matvec_dot<T>(const Geo&, const Coef<T>&, const T*, T*, double*,   \
                                          cudaStream_t, FinSpec);                              \
    template int64_t launch_update_xr<T>(int64_t, const Scal*, const T*, const T*, T*, T*,     \
                                         double*, cudaStream_t, FinSpec, bool);                \
    template int64_t launch_update_r<T>(int64_t, const Scal*, const T*, T*, double*,           \
                                        cudaStream_t, FinSpec, bool);                          \
    template int64_t launch_dot2<T>(int64_t, const T*, const T*, const T*, double*,            \
                                    cudaStream_t, FinSpec, bool);                              \
    template void launch_xpby<T>(int64_t, const Scal*, const T*, T*, cudaStream_t);

PARIS_INSTANTIATE(float)
PARIS_INSTANTIATE(double)

}  // namespace paris
