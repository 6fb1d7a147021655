// Batched projection: many independent projection steps of uneven grid sizes
// in ONE persistent cooperative launch.
//
// Each instance is the full projection step of the single-grid path (face
// coefficients, divergence and mean removal, multigrid hierarchy set-up,
// FP64 iterative refinement around FP32 flexible CG preconditioned by a
// red-black V-cycle with an FP64 dense coarsest solve, mean removal of p,
// velocity correction), run on the device by a group of CTAs sized in
// proportion to the instance's cells.  The groups never wait for one another:
// inside a group, phases are separated by a group barrier (an atomic counter
// and a generation word in global memory, spun on with an iteration limit
// after which the kernel records an error and returns), and per-instance
// reductions are folded by every CTA of the group in the same fixed order, so
// all of them take the same decisions.  The launch is cooperative, which
// guarantees that every CTA is resident, so a group barrier always completes.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/paris.h"
#include "kernels.cuh"

namespace paris {
namespace batch {

constexpr int kBT = 256;     // threads per CTA
constexpr int kMaxLev = 12;  // multigrid levels per instance
constexpr int kMaxDense = 128;

struct BLevel {
    Geo g;
    int fac[3];
    float* b[3];  // coefficients beta/h_a^2 of this level
    float* x;     // level solution (level 0: the V-cycle output)
    float* f;     // level right-hand side (level 0: the V-cycle input)
};

struct BInst {
    Geo g0;
    double h, dt, rho1, rho2;
    int nlev, ncoarse, dense;
    BLevel lv[kMaxLev];
    const double* C;
    double *u, *v, *w, *p;
    double* b64[3];  // FP64 face coefficients
    double* f64;     // right-hand side of A p = f (negated, mean-free)
    float *r, *z, *d, *q, *e;
    double* cinv;  // dense inverse of the regularised coarsest operator
    int cta0, ncta;
    unsigned* bar;  // group barrier: [0] arrivals, [1] generation
    double* part;   // group partials: 2 buffers x ncta x 4
    double* stats;  // 8 values (see write_stats)
};

struct BParams {
    double tol, inner_tol;
    int max_iter, nu1, nu2;
    float omega;
    long long spin_limit;
};

// ------------------------------------------------------------ group ops ---

struct Grp {
    const BInst* I;
    int rank, ncta;
    int* err;
    int pb;
    long long spin;
};

__device__ inline bool group_ok(const Grp& c) { return *(volatile int*)c.err == 0; }

// Barrier of the instance's CTAs (bounded spin).  Returns false once any
// barrier of the launch has timed out, so that every CTA unwinds.
__device__ bool gbar(Grp& c) {
    __syncthreads();
    if (c.ncta > 1) {
        if (threadIdx.x == 0) {
            volatile unsigned* gen = c.I->bar + 1;
            const unsigned g = *gen;
            __threadfence();
            const unsigned arrived = atomicAdd(c.I->bar, 1u);
            if (arrived == (unsigned)c.ncta - 1) {
                c.I->bar[0] = 0;
                __threadfence();
                atomicAdd(c.I->bar + 1, 1u);
            } else {
                long long it = 0;
                while (*gen == g) {
                    if (++it > c.spin || *(volatile int*)c.err) {
                        atomicExch(c.err, 1);
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
        }
        __syncthreads();
    }
    return group_ok(c);
}

// Sum (op 0) or max (op 1) of NV values over the instance, identical in all
// of its CTAs (fixed folding order).
template <int NV>
__device__ bool greduce(Grp& c, double (&v)[NV], const int (&op)[NV]) {
    __shared__ double sh[kBT / 32][4];
    __shared__ double res[4];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double t = op[q] ? warp_max(v[q]) : warp_sum(v[q]);
        if (lane == 0) sh[wid][q] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 0; q < NV; ++q) {
            double t = 0.0;
            for (int w = 0; w < kBT / 32; ++w) t = op[q] ? fmax(t, sh[w][q]) : t + sh[w][q];
            res[q] = t;
            if (c.ncta > 1) c.I->part[((int64_t)c.pb * c.ncta + c.rank) * 4 + q] = t;
        }
    }
    if (c.ncta > 1) {
        if (!gbar(c)) return false;
        if (threadIdx.x == 0) {
            for (int q = 0; q < NV; ++q) {
                double t = 0.0;
                for (int r = 0; r < c.ncta; ++r) {
                    const double x = *(volatile double*)&c.I->part[((int64_t)c.pb * c.ncta + r) * 4 + q];
                    t = op[q] ? fmax(t, x) : t + x;
                }
                res[q] = t;
            }
        }
        c.pb ^= 1;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = res[q];
    __syncthreads();
    return group_ok(c);
}

#define GLOOP(c_, n_)                                                          \
    for (int64_t c_ = (int64_t)cx.rank * kBT + threadIdx.x; c_ < (int64_t)(n_); \
         c_ += (int64_t)cx.ncta * kBT)

// cell index -> (i, j, k) in 32-bit arithmetic (an instance has fewer than
// 2^31 cells and faces, checked at creation)
__device__ inline void decomp(const Geo& g, int64_t c, int& i, int& j, int& k) {
    const unsigned cu = (unsigned)c, nx = (unsigned)g.nx, ny = (unsigned)g.ny;
    const unsigned t = cu / nx;
    i = (int)(cu - t * nx);
    k = (int)(t / ny);
    j = (int)(t - (unsigned)k * ny);
}

// ------------------------------------------------------------ set-up ---

// beta_f = 2/(rho_L + rho_R), rho = rho1 C + rho2 (1 - C) (Eq. muH), 0 on walls;
// FP64 for the residual and the correction, FP32 beta/h^2 for the V-cycle.
__device__ void setup_coefficients(Grp& cx) {
    const BInst& I = *cx.I;
    const Geo& g = I.g0;
    const double ih2 = 1.0 / (I.h * I.h);
    auto rho = [&](double cc) { return fma(I.rho1, cc, I.rho2 * (1.0 - cc)); };
    GLOOP(c, g.ncell()) {
        int i, j, k;
        decomp(g, c, i, j, k);
        const double rc = rho(I.C[c]);
        AxisNb ax = axis_nb(i, g.nx, g.wx), ay = axis_nb(j, g.ny, g.wy), az = axis_nb(k, g.nz, g.wz);
        auto put = [&](int a, int64_t f, bool wall, int64_t left) {
            const double bt = wall ? 0.0 : 2.0 / (rho(I.C[left]) + rc);
            I.b64[a][f] = bt;
            I.lv[0].b[a][f] = (float)(bt * ih2);
        };
        put(0, g.fx(i, j, k), ax.wm, g.cidx(ax.m, j, k));
        put(1, g.fy(i, j, k), ay.wm, g.cidx(i, ay.m, k));
        put(2, g.fz(i, j, k), az.wm, g.cidx(i, j, az.m));
        if (g.wx && i == g.nx - 1) { I.b64[0][g.fx(g.nx, j, k)] = 0.0; I.lv[0].b[0][g.fx(g.nx, j, k)] = 0.f; }
        if (g.wy && j == g.ny - 1) { I.b64[1][g.fy(i, g.ny, k)] = 0.0; I.lv[0].b[1][g.fy(i, g.ny, k)] = 0.f; }
        if (g.wz && k == g.nz - 1) { I.b64[2][g.fz(i, j, g.nz)] = 0.0; I.lv[0].b[2][g.fz(i, j, g.nz)] = 0.f; }
    }
}

// f = -(div u*/dt - mean) and its norms; returns false on error
__device__ bool setup_rhs(Grp& cx, double& bnorm2, double& binf, double& nonfin) {
    const BInst& I = *cx.I;
    const Geo& g = I.g0;
    const double ihdt = 1.0 / (I.h * I.dt);
    double acc[1] = {0.0};
    GLOOP(c, g.ncell()) {
        int i, j, k;
        decomp(g, c, i, j, k);
        AxisNb ax = axis_nb(i, g.nx, g.wx), ay = axis_nb(j, g.ny, g.wy), az = axis_nb(k, g.nz, g.wz);
        const double up = ax.wp ? 0.0 : I.u[g.fx(ax.fp, j, k)], um = ax.wm ? 0.0 : I.u[g.fx(i, j, k)];
        const double vp = ay.wp ? 0.0 : I.v[g.fy(i, ay.fp, k)], vm = ay.wm ? 0.0 : I.v[g.fy(i, j, k)];
        const double wp = az.wp ? 0.0 : I.w[g.fz(i, j, az.fp)], wm = az.wm ? 0.0 : I.w[g.fz(i, j, k)];
        const double b = (((up - um) + (vp - vm)) + (wp - wm)) * ihdt;
        I.f64[c] = b;
        acc[0] += b;
    }
    const int op1[1] = {0};
    if (!greduce<1>(cx, acc, op1)) return false;
    const double mean = acc[0] / (double)g.ncell();
    double n3[3] = {0.0, 0.0, 0.0};
    unsigned nf = 0;
    GLOOP(c, g.ncell()) {
        const double t = -(I.f64[c] - mean);
        I.f64[c] = t;
        I.p[c] = 0.0;
        n3[0] = fma(t, t, n3[0]);
        n3[1] = fmax(n3[1], fabs(t));
        nf += isfinite(t) ? 0u : 1u;
    }
    n3[2] = (double)nf;
    const int op3[3] = {0, 1, 0};
    if (!greduce<3>(cx, n3, op3)) return false;
    bnorm2 = n3[0];
    binf = n3[1];
    nonfin = n3[2];
    return true;
}

// coarse coefficients: mean of the covering fine faces times (h_f/h_c)^2
__device__ bool setup_levels(Grp& cx) {
    const BInst& I = *cx.I;
    for (int l = 1; l < I.nlev; ++l) {
        const BLevel& F = I.lv[l - 1];
        const BLevel& L = I.lv[l];
        for (int a = 0; a < 3; ++a) {
            const int n0 = L.g.nx + (a == 0 ? L.g.wx : 0), n1 = L.g.ny + (a == 1 ? L.g.wy : 0);
            const int fn0 = F.g.nx + (a == 0 ? F.g.wx : 0), fn1 = F.g.ny + (a == 1 ? F.g.wy : 0);
            const float ratio = 1.0f / (float)(L.fac[a] * L.fac[a]);
            GLOOP(t, L.g.nface(a)) {
                const int C3[3] = {(int)(t % n0), (int)((t / n0) % n1), (int)(t / ((int64_t)n0 * n1))};
                int lo[3], cnt[3];
                for (int b = 0; b < 3; ++b) {
                    lo[b] = C3[b] * L.fac[b];
                    cnt[b] = b == a ? 1 : L.fac[b];
                }
                float s = 0.f;
                for (int dk = 0; dk < cnt[2]; ++dk)
                    for (int dj = 0; dj < cnt[1]; ++dj)
                        for (int di = 0; di < cnt[0]; ++di)
                            s += F.b[a][((int64_t)(lo[2] + dk) * fn1 + (lo[1] + dj)) * fn0 + (lo[0] + di)];
                L.b[a][t] = s / (float)(cnt[0] * cnt[1] * cnt[2]) * ratio;
            }
        }
        if (!gbar(cx)) return false;
    }
    // dense inverse of the coarsest operator (FP64 Gauss-Jordan by the first CTA)
    if (I.dense && cx.rank == 0) {
        const BLevel& L = I.lv[I.nlev - 1];
        const int n = I.ncoarse;
        double* M = I.cinv;
        for (int e = threadIdx.x; e < n * n; e += kBT) M[e] = 0.0;
        __syncthreads();
        for (int c = threadIdx.x; c < n; c += kBT) {
            const int i = c % L.g.nx, j = (c / L.g.nx) % L.g.ny, k = c / (L.g.nx * L.g.ny);
            Coef<float> cf{L.b[0], L.b[1], L.b[2], 1.0f};
            Stencil<float> s;
            int c32_;
            load_stencil_fast(L.g, cf.bx, cf.by, cf.bz, i, j, k, s, c32_);
            for (int q = 0; q < 6; ++q) {
                M[(int64_t)c * n + c] += (double)s.b[q];
                M[(int64_t)c * n + s.nb[q]] -= (double)s.b[q];
            }
        }
        __syncthreads();
        __shared__ double dsum, piv;
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int c = 0; c < n; ++c) t += M[(int64_t)c * n + c];
            dsum = t / ((double)n * (double)n);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < n * n; e += kBT) M[e] += dsum;
        __syncthreads();
        __shared__ double col[kMaxDense];
        for (int kk = 0; kk < n; ++kk) {
            if (threadIdx.x == 0) piv = 1.0 / M[(int64_t)kk * n + kk];
            for (int r = threadIdx.x; r < n; r += kBT) col[r] = M[(int64_t)r * n + kk];
            __syncthreads();
            for (int cc = threadIdx.x; cc < n; cc += kBT)
                M[(int64_t)kk * n + cc] = (cc == kk) ? piv : M[(int64_t)kk * n + cc] * piv;
            __syncthreads();
            for (int e = threadIdx.x; e < n * n; e += kBT) {
                const int r = e / n, cc = e % n;
                if (r == kk) continue;
                if (cc == kk) M[e] = -col[r] * piv;
                else M[e] -= col[r] * M[(int64_t)kk * n + cc];
            }
            __syncthreads();
        }
    }
    return gbar(cx);
}

// ------------------------------------------------------------ V-cycle ---

// The colour-c cell of pair pp of a level (i >= nx: none; io: the other
// member of the pair, or nx when it does not exist).
struct PassCell {
    int i, j, k, io;
};
__device__ inline PassCell pass_cell(const Geo& g, unsigned pp, unsigned npair, int color) {
    const unsigned ny = (unsigned)g.ny, row = pp / npair;
    PassCell p;
    const int tp = (int)(pp - row * npair);
    p.k = (int)(row / ny);
    p.j = (int)(row - (unsigned)p.k * ny);
    const int i0 = 2 * tp;
    p.i = i0 + ((i0 + p.j + p.k + color) & 1);
    p.io = 2 * i0 + 1 - p.i;
    return p;
}

// The loaded values of one pass cell: face coefficients, f, x and the
// neighbours' x.
struct PassLoad {
    float b[6];
    int c;
    float f, x, nb[6];
    bool on;
};
__device__ __forceinline__ void pass_load(PassLoad& d, const BLevel& L, const float* f, const float* x,
                                          const PassCell& p, bool zero) {
    d.on = p.i < L.g.nx;
    if (!d.on) return;
    Stencil<float> s;
    load_stencil_fast(L.g, L.b[0], L.b[1], L.b[2], p.i, p.j, p.k, s, d.c);
#pragma unroll
    for (int q = 0; q < 6; ++q) d.b[q] = s.b[q];
    d.f = f[d.c];
    if (!zero) {
        d.x = x[d.c];
#pragma unroll
        for (int q = 0; q < 6; ++q) d.nb[q] = x[(int)s.nb[q]];
    }
}
__device__ __forceinline__ void pass_store(const PassLoad& d, const Geo& g, float* x, const PassCell& p,
                                           float omega, bool zero) {
    if (zero && p.io < g.nx) x[g.cidx(p.io, p.j, p.k)] = 0.f;
    if (!d.on) return;
    const float sum = ((d.b[0] + d.b[1]) + (d.b[2] + d.b[3])) + (d.b[4] + d.b[5]);
    const float wv = sum > 0.f ? 1.f / sum : 0.f;
    if (zero) {
        x[d.c] = omega * wv * d.f;
    } else {
        float acc = d.f;
#pragma unroll
        for (int q = 0; q < 6; ++q) acc = fmaf(d.b[q], d.nb[q], acc);
        x[d.c] = fmaf(omega, fmaf(wv, acc, -d.x), d.x);
    }
}

// One red-black colour pass in place on level L (zero: x taken as 0 and the
// other colour zeroed).  x_c <- x_c + omega (w (f + sum beta x_nb) - x_c).
// A thread takes two pairs per iteration and loads both stencils before it
// updates either: cells of the updated colour are never neighbours of one
// another, so the two updates are independent.
__device__ __noinline__ void rb_pass(Grp& cx, const BLevel& L, const float* f, float* x, int color, float omega,
                        bool zero) {
    const Geo& g = L.g;
    const unsigned npair = (unsigned)(g.nx + 1) / 2;
    const int64_t total = (int64_t)npair * g.ny * g.nz;
    const int64_t stride = (int64_t)cx.ncta * kBT;
    for (int64_t p0 = (int64_t)cx.rank * kBT + threadIdx.x; p0 < total; p0 += 2 * stride) {
        const int64_t p1 = p0 + stride;
        const PassCell a = pass_cell(g, (unsigned)p0, npair, color);
        const PassCell b = p1 < total ? pass_cell(g, (unsigned)p1, npair, color) : PassCell{g.nx, 0, 0, g.nx};
        PassLoad da, db;
        pass_load(da, L, f, x, a, zero);
        pass_load(db, L, f, x, b, zero);
        pass_store(da, g, x, a, omega, zero);
        pass_store(db, g, x, b, omega, zero);
    }
}

__device__ bool vcycle(Grp& cx, const BParams& P, const float* f0, float* x0) {
    const BInst& I = *cx.I;
    const int nl = I.nlev;
    for (int l = 0; l < nl - 1; ++l) {
        const BLevel& L = I.lv[l];
        const float* f = l == 0 ? f0 : L.f;
        float* x = l == 0 ? x0 : L.x;
        for (int s = 0; s < P.nu1; ++s) {
            rb_pass(cx, L, f, x, 0, P.omega, s == 0);
            if (!gbar(cx)) return false;
            rb_pass(cx, L, f, x, 1, P.omega, false);
            if (!gbar(cx)) return false;
        }
        if (P.nu1 == 0) {
            GLOOP(c, L.g.ncell()) x[c] = 0.f;
            if (!gbar(cx)) return false;
        }
        const BLevel& Cl = I.lv[l + 1];
        Coef<float> cf{L.b[0], L.b[1], L.b[2], 1.0f};
        GLOOP(cc, Cl.g.ncell()) {
            int I0, J0, K0;
            decomp(Cl.g, cc, I0, J0, K0);
            float sum = 0.f;
            for (int dk = 0; dk < Cl.fac[2]; ++dk)
                for (int dj = 0; dj < Cl.fac[1]; ++dj)
                    for (int di = 0; di < Cl.fac[0]; ++di) {
                        const int i = I0 * Cl.fac[0] + di, j = J0 * Cl.fac[1] + dj, k = K0 * Cl.fac[2] + dk;
                        const int64_t c = L.g.cidx(i, j, k);
                        Stencil<float> s;
                        int c32_;
                        load_stencil_fast(L.g, cf.bx, cf.by, cf.bz, i, j, k, s, c32_);
                        sum += f[c] - apply_A(s, x, x[c], 1.0f);
                    }
            Cl.f[cc] = sum / (float)(Cl.fac[0] * Cl.fac[1] * Cl.fac[2]);
        }
        if (!gbar(cx)) return false;
    }
    {
        const BLevel& Cl = I.lv[nl - 1];
        const float* f = nl == 1 ? f0 : Cl.f;
        float* x = nl == 1 ? x0 : Cl.x;
        if (I.dense) {
            if (cx.rank == 0) {
                const int n = I.ncoarse;
                __shared__ double fs[kMaxDense];
                __shared__ double mean;
                for (int c = threadIdx.x; c < n; c += kBT) fs[c] = (double)f[c];
                __syncthreads();
                if (threadIdx.x == 0) {
                    double t = 0.0;
                    for (int c = 0; c < n; ++c) t += fs[c];
                    mean = t / n;
                }
                __syncthreads();
                for (int r = threadIdx.x; r < n; r += kBT) {
                    double acc = 0.0;
                    for (int c = 0; c < n; ++c) acc = fma(I.cinv[(int64_t)r * n + c], fs[c] - mean, acc);
                    x[r] = (float)acc;
                }
            }
            if (!gbar(cx)) return false;
        } else {
            for (int s = 0; s < 8; ++s) {
                rb_pass(cx, Cl, f, x, 0, P.omega, s == 0);
                if (!gbar(cx)) return false;
                rb_pass(cx, Cl, f, x, 1, P.omega, false);
                if (!gbar(cx)) return false;
            }
            for (int s = 0; s < 8; ++s) {
                rb_pass(cx, Cl, f, x, 1, P.omega, false);
                if (!gbar(cx)) return false;
                rb_pass(cx, Cl, f, x, 0, P.omega, false);
                if (!gbar(cx)) return false;
            }
        }
    }
    for (int l = nl - 2; l >= 0; --l) {
        const BLevel& L = I.lv[l];
        const BLevel& Cl = I.lv[l + 1];
        const float* f = l == 0 ? f0 : L.f;
        float* x = l == 0 ? x0 : L.x;
        GLOOP(c, L.g.ncell()) {
            int i, j, k;
            decomp(L.g, c, i, j, k);
            // coarsening factors are 1 or 2: halving is a shift
            x[c] += Cl.x[Cl.g.cidx(i >> (Cl.fac[0] - 1), j >> (Cl.fac[1] - 1), k >> (Cl.fac[2] - 1))];
        }
        if (!gbar(cx)) return false;
        for (int s = 0; s < P.nu2; ++s) {
            rb_pass(cx, L, f, x, 1, P.omega, false);
            if (!gbar(cx)) return false;
            rb_pass(cx, L, f, x, 0, P.omega, false);
            if (!gbar(cx)) return false;
        }
    }
    return true;
}

// ------------------------------------------------------------ solve ---

__device__ bool solve(Grp& cx, const BParams& P, double bnorm2, double binf, int& iters, int& outer,
                      double& rr, double& rinf, int& converged) {
    const BInst& I = *cx.I;
    const Geo& g = I.g0;
    const int64_t N = g.ncell();
    Coef<double> c64{I.b64[0], I.b64[1], I.b64[2], 1.0 / (I.h * I.h)};
    Coef<float> c32{I.lv[0].b[0], I.lv[0].b[1], I.lv[0].b[2], 1.0f};
    const double tol = P.tol;
    double rinf_prev = binf, prev_rr = INFINITY;
    int stalls = 0;
    iters = outer = converged = 0;
    rr = bnorm2;
    rinf = binf;
    if (bnorm2 == 0.0) {
        converged = 1;
        return true;
    }
    for (;;) {
        // FP64 true residual, scaled FP32 copy for the inner solve
        const double scale = 1.0 / (rinf_prev > 1e-300 ? rinf_prev : 1.0);
        double n3[3] = {0.0, 0.0, 0.0};
        unsigned nonfin = 0;
        GLOOP(c, N) {
            int i, j, k;
            decomp(g, c, i, j, k);
            Stencil<double> s;
            int c32_;
            load_stencil_fast(g, c64.bx, c64.by, c64.bz, i, j, k, s, c32_);
            const double r = I.f64[c] - apply_A(s, I.p, I.p[c], c64.scale);
            I.r[c] = (float)(r * scale);
            n3[0] = fma(r, r, n3[0]);
            n3[1] = fmax(n3[1], fabs(r));
            nonfin += isfinite(r) ? 0u : 1u;
        }
        n3[2] = (double)nonfin;
        const int op3[3] = {0, 1, 0};
        if (!greduce<3>(cx, n3, op3)) return false;
        rr = n3[0];
        rinf = n3[1];
        if (n3[2] > 0) return true;
        if (rr <= tol * tol * bnorm2 && rinf <= tol * binf) {
            converged = 1;
            return true;
        }
        if (iters >= P.max_iter) return true;
        if (rr > 0.25 * prev_rr) {
            if (++stalls >= 2) return true;
        } else {
            stalls = 0;
        }
        prev_rr = rr;
        ++outer;
        const double rr32 = rr * scale * scale;
        double need2 = (tol * tol * bnorm2) / fmax(rr, 1e-300) * 1e-2;
        const double target = rr32 * fmax(P.inner_tol * P.inner_tol, fmin(need2, 1.0));
        // inner flexible CG on A e = r (FP32 vectors, FP64 group sums)
        GLOOP(c, N) I.e[c] = 0.f;
        if (!vcycle(cx, P, I.r, I.z)) return false;
        // per-thread sums in FP32 (the element-wise products' precision),
        // across threads and CTAs in FP64
        float a0 = 0.f;
        GLOOP(c, N) {
            a0 = fmaf(I.r[c], I.z[c], a0);
            I.d[c] = I.z[c];
        }
        double d2[2] = {(double)a0, 0.0};
        const int op2[2] = {0, 0};
        if (!greduce<2>(cx, d2, op2)) return false;
        double rho = d2[0];
        for (int jj = 0; jj < 50 && iters < P.max_iter; ++jj) {
            float aq = 0.f;
            GLOOP(c, N) {
                int i, j, k;
                decomp(g, c, i, j, k);
                Stencil<float> s;
                int c32_;
                load_stencil_fast(g, c32.bx, c32.by, c32.bz, i, j, k, s, c32_);
                const float qc = apply_A(s, I.d, I.d[c], 1.0f);
                I.q[c] = qc;
                aq = fmaf(I.d[c], qc, aq);
            }
            double dq[1] = {(double)aq};
            const int op1[1] = {0};
            if (!greduce<1>(cx, dq, op1)) return false;
            const double alpha = dq[0] > 0.0 ? rho / dq[0] : 0.0;
            const float af = (float)alpha;
            float ar = 0.f;
            unsigned nonfin = 0;
            GLOOP(c, N) {
                I.e[c] = fmaf(af, I.d[c], I.e[c]);
                const float rc = fmaf(-af, I.q[c], I.r[c]);
                I.r[c] = rc;
                ar = fmaf(rc, rc, ar);
                nonfin += isfinite(rc) ? 0u : 1u;
            }
            double rn[2] = {(double)ar, (double)nonfin};
            if (!greduce<2>(cx, rn, op2)) return false;
            ++iters;
            if (rn[1] > 0 || rn[0] <= target || rn[0] > 1e6 * rr32) break;
            if (!vcycle(cx, P, I.r, I.z)) return false;
            float z0 = 0.f, z1 = 0.f;
            GLOOP(c, N) {
                z0 = fmaf(I.z[c], I.r[c], z0);
                z1 = fmaf(I.z[c], I.q[c], z1);
            }
            double zz[2] = {(double)z0, (double)z1};
            if (!greduce<2>(cx, zz, op2)) return false;
            const double beta = rho != 0.0 ? -alpha * zz[1] / rho : 0.0;
            rho = zz[0];
            const float bf = (float)beta;
            GLOOP(c, N) I.d[c] = fmaf(bf, I.d[c], I.z[c]);
            if (!gbar(cx)) return false;
        }
        const double inv = 1.0 / scale;
        GLOOP(c, N) I.p[c] = fma((double)I.e[c], inv, I.p[c]);
        if (!gbar(cx)) return false;
        rinf_prev = rinf;
    }
}

__global__ void __launch_bounds__(kBT, 2) persistent_kernel(const BInst* __restrict__ insts,
                                                         const int* __restrict__ cta_inst,
                                                         BParams P, int* err) {
    Grp cx;
    const int inst = cta_inst[blockIdx.x];
    if (inst < 0) return;  // spare CTA
    cx.I = &insts[inst];
    cx.rank = blockIdx.x - cx.I->cta0;
    cx.ncta = cx.I->ncta;
    cx.err = err;
    cx.pb = 0;
    cx.spin = P.spin_limit;
    const BInst& I = *cx.I;
    double bnorm2 = 0, binf = 0, nonfin = 0, rr = 0, rinf = 0;
    int iters = 0, outer = 0, converged = 0;
    setup_coefficients(cx);
    if (!gbar(cx)) return;
    if (!setup_rhs(cx, bnorm2, binf, nonfin)) return;
    if (!setup_levels(cx)) return;
    if (nonfin == 0) {
        if (!solve(cx, P, bnorm2, binf, iters, outer, rr, rinf, converged)) return;
    }
    // mean-free p, then u = u* - dt beta grad p (walls blocked)
    double m[1] = {0.0};
    GLOOP(c, I.g0.ncell()) m[0] += I.p[c];
    const int op1[1] = {0};
    if (!greduce<1>(cx, m, op1)) return;
    const double mean = m[0] / (double)I.g0.ncell();
    GLOOP(c, I.g0.ncell()) I.p[c] -= mean;
    if (!gbar(cx)) return;
    const Geo& g = I.g0;
    const double dth = I.dt / I.h;
    GLOOP(c, g.ncell()) {
        int i, j, k;
        decomp(g, c, i, j, k);
        const double pc = I.p[c];
        AxisNb ax = axis_nb(i, g.nx, g.wx), ay = axis_nb(j, g.ny, g.wy), az = axis_nb(k, g.nz, g.wz);
        int64_t f = g.fx(i, j, k);
        I.u[f] = ax.wm ? 0.0 : I.u[f] - dth * I.b64[0][f] * (pc - I.p[g.cidx(ax.m, j, k)]);
        f = g.fy(i, j, k);
        I.v[f] = ay.wm ? 0.0 : I.v[f] - dth * I.b64[1][f] * (pc - I.p[g.cidx(i, ay.m, k)]);
        f = g.fz(i, j, k);
        I.w[f] = az.wm ? 0.0 : I.w[f] - dth * I.b64[2][f] * (pc - I.p[g.cidx(i, j, az.m)]);
        if (g.wx && i == g.nx - 1) I.u[g.fx(g.nx, j, k)] = 0.0;
        if (g.wy && j == g.ny - 1) I.v[g.fy(i, g.ny, k)] = 0.0;
        if (g.wz && k == g.nz - 1) I.w[g.fz(i, j, g.nz)] = 0.0;
    }
    if (cx.rank == 0 && threadIdx.x == 0) {
        I.stats[0] = iters;
        I.stats[1] = outer;
        I.stats[2] = bnorm2 > 0 ? sqrt(rr / bnorm2) : 0.0;
        I.stats[3] = binf > 0 ? rinf / binf : 0.0;
        I.stats[4] = converged;
        I.stats[5] = nonfin;
        I.stats[6] = I.nlev;
        I.stats[7] = 1.0;  // finished
    }
}

}  // namespace batch
}  // namespace paris

// ==================================================================== host ===

using namespace paris;
using namespace paris::batch;

namespace {

struct HostInst {
    paris_grid grid;
    Geo g0;
    std::vector<Geo> lev;
    std::vector<std::array<int, 3>> fac;
    int64_t cell_off, face_off[3];
};

std::vector<std::pair<Geo, std::array<int, 3>>> plan(const Geo& g0, int coarse_max) {
    std::vector<std::pair<Geo, std::array<int, 3>>> out;
    out.push_back({g0, {1, 1, 1}});
    while ((int)out.size() < kMaxLev) {
        Geo c = out.back().first;
        if (c.ncell() <= coarse_max) break;
        int n[3] = {c.nx, c.ny, c.nz};
        bool can[3], all = true, any = false;
        for (int a = 0; a < 3; ++a) {
            can[a] = n[a] % 2 == 0 && n[a] >= 4;
            all = all && can[a];
            any = any || can[a];
        }
        if (!any) break;
        std::array<int, 3> f{};
        for (int a = 0; a < 3; ++a) {
            f[a] = (all || can[a]) ? 2 : 1;
            n[a] /= f[a];
        }
        c.nx = n[0];
        c.ny = n[1];
        c.nz = n[2];
        out.push_back({c, f});
    }
    return out;
}

}  // namespace

struct paris_batch {
    int n = 0;
    paris_opts opts;
    cudaStream_t st = nullptr;    // the batch's own stream (capturable)
    cudaStream_t user = nullptr;  // the caller's stream: work there is ordered before each step
    cudaEvent_t ev = nullptr;
    std::vector<HostInst> hi;
    int64_t cells = 0, faces[3] = {0, 0, 0};
    // device
    std::vector<void*> allocs;
    BInst* d_inst = nullptr;
    int* d_cta = nullptr;
    int* d_err = nullptr;
    double* d_stats = nullptr;
    unsigned* d_bar = nullptr;
    double* d_part = nullptr;  // group partials: 2 x 4 doubles per CTA of the largest launch
    int max_ctas = 0;
    std::vector<BInst> h_inst;  // host copy of the descriptors
    double* h_stats = nullptr;  // pinned
    int grid = 0, bps = 0;      // CTAs in the launch, CTAs per SM
    BParams prm{};
    // CUDA graph of one step (rebuilt when the pools change)
    cudaGraphExec_t exec = nullptr;
    const void* graph_key[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    double* h_scalars = nullptr;  // pinned: rho1, rho2, dt per instance
    double* d_scalars = nullptr;
};

namespace {

template <typename T>
T* balloc(paris_batch* b, int64_t n, cudaError_t& e) {
    void* p = nullptr;
    if (e != cudaSuccess) return nullptr;
    e = cudaMalloc(&p, std::max<int64_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) b->allocs.push_back(p);
    return (T*)p;
}

// CTA allotment in proportion to the cells, at least one CTA per instance.
std::vector<int> allot(const std::vector<int64_t>& work, int R) {
    const int n = (int)work.size();
    double tot = 0;
    for (auto w : work) tot += (double)w;
    std::vector<int> k(n, 1);
    int used = n;
    // greedy: give the next CTA to the instance with the most cells per CTA
    while (used < R) {
        int best = -1;
        double bw = 0;
        for (int i = 0; i < n; ++i) {
            const int64_t cap = std::max<int64_t>(1, work[i] / (kBT * 4));
            if (k[i] >= cap) continue;
            const double w = (double)work[i] / k[i];
            if (w > bw) { bw = w; best = i; }
        }
        if (best < 0) break;
        ++k[best];
        ++used;
    }
    return k;
}

paris_status build_descriptors(paris_batch* b) {
    cudaError_t e = cudaSuccess;
    // launch size: every CTA must be resident (cooperative launch)
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_kernel, kBT, 0);
    if (per_sm < 1 || sms < 1) return PARIS_ERR_CUDA;
    b->bps = std::min(per_sm, std::max(1, b->bps > 0 ? b->bps : per_sm));
    const int R = sms * b->bps;
    if (R < b->n) return PARIS_ERR_INVALID_ARG;  // one CTA per instance at least
    std::vector<int64_t> work(b->n);
    for (int i = 0; i < b->n; ++i) work[i] = b->hi[i].g0.ncell();
    std::vector<int> k = allot(work, R);
    std::vector<int> cta(R, -1);
    int pos = 0;
    for (int i = 0; i < b->n; ++i) {
        b->h_inst[i].cta0 = pos;
        b->h_inst[i].ncta = k[i];
        for (int q = 0; q < k[i]; ++q) cta[pos++] = i;
    }
    b->grid = R;
    if (!b->d_cta) b->d_cta = balloc<int>(b, b->max_ctas, e);
    if (e != cudaSuccess) return PARIS_ERR_NO_MEMORY;
    // each instance's partial-sum slots: 2 buffers x 4 values x its CTAs
    if (R > b->max_ctas) return PARIS_ERR_INVALID_ARG;
    for (int i = 0; i < b->n; ++i) {
        b->h_inst[i].part = b->d_part + (int64_t)8 * b->h_inst[i].cta0;
        b->h_inst[i].bar = b->d_bar + 2 * i;
        b->h_inst[i].stats = b->d_stats + 8 * i;
    }
    if (cudaMemcpy(b->d_cta, cta.data(), sizeof(int) * R, cudaMemcpyHostToDevice) != cudaSuccess)
        return PARIS_ERR_CUDA;
    return PARIS_OK;
}

void set_params(paris_batch* b) {
    b->prm.tol = b->opts.tol;
    b->prm.inner_tol = b->opts.inner_tol;
    b->prm.max_iter = b->opts.max_iter;
    b->prm.nu1 = b->opts.nu1;
    b->prm.nu2 = b->opts.nu2;
    b->prm.omega = (float)b->opts.omega;
    b->prm.spin_limit = 1ll << 24;  // ~2 s at 64 ns per spin
}

}  // namespace

// The per-instance scalars are copied into the descriptors at every step.
__global__ void batch_scalars_kernel(int n, const double* s, BInst* inst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    inst[i].rho1 = s[3 * i];
    inst[i].rho2 = s[3 * i + 1];
    inst[i].dt = s[3 * i + 2];
}

extern "C" {

paris_status paris_batch_create(paris_batch** out, int n, const paris_grid* grids,
                                const paris_opts* o, void* stream) {
    if (!out || n < 1 || !grids) return PARIS_ERR_INVALID_ARG;
    *out = nullptr;
    paris_opts def;
    paris_default_opts(&def);
    if (!o) o = &def;
    if (o->smoother != PARIS_SMOOTH_RBGS && o->smoother != PARIS_SMOOTH_RBGS_2PASS) return PARIS_ERR_INVALID_ARG;
    if (!(o->tol > 0) || o->max_iter < 1 || o->nu1 < 0 || o->nu2 < 0 || o->nu1 + o->nu2 < 1 ||
        !(o->omega > 0 && o->omega < 2) || o->coarse_max_cells < 1 || o->coarse_max_cells > kMaxDense ||
        !(o->inner_tol > 0 && o->inner_tol < 1))
        return PARIS_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        const paris_grid& g = grids[i];
        if (g.nx < 2 || g.ny < 2 || g.nz < 2 || !(g.h > 0)) return PARIS_ERR_INVALID_ARG;
        for (int a = 0; a < 3; ++a)
            if (g.bc[a] != PARIS_PERIODIC && g.bc[a] != PARIS_WALL) return PARIS_ERR_INVALID_ARG;
        // every array of an instance is indexed in 32 bits on the device
        if ((int64_t)(g.nx + 1) * (g.ny + 1) * (g.nz + 1) >= ((int64_t)1 << 31)) return PARIS_ERR_INVALID_ARG;
    }
    paris_batch* b = new (std::nothrow) paris_batch();
    if (!b) return PARIS_ERR_NO_MEMORY;
    b->n = n;
    b->opts = *o;
    b->user = (cudaStream_t)stream;
    // the legacy default stream cannot be captured into a graph: the batch
    // runs on its own stream, ordered after the caller's by an event
    if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) {
        delete b;
        return PARIS_ERR_CUDA;
    }
    b->hi.resize(n);
    b->h_inst.assign(n, BInst{});
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n; ++i) {
        HostInst& H = b->hi[i];
        H.grid = grids[i];
        H.g0 = Geo{grids[i].nx, grids[i].ny, grids[i].nz, grids[i].bc[0] == PARIS_WALL,
                   grids[i].bc[1] == PARIS_WALL, grids[i].bc[2] == PARIS_WALL};
        H.cell_off = b->cells;
        b->cells += H.g0.ncell();
        for (int a = 0; a < 3; ++a) {
            H.face_off[a] = b->faces[a];
            b->faces[a] += H.g0.nface(a);
        }
        auto lv = plan(H.g0, o->coarse_max_cells);
        BInst& I = b->h_inst[i];
        I.g0 = H.g0;
        I.h = grids[i].h;
        I.nlev = (int)lv.size();
        I.ncoarse = (int)lv.back().first.ncell();
        I.dense = I.ncoarse <= kMaxDense;
        for (int l = 0; l < I.nlev; ++l) {
            BLevel& L = I.lv[l];
            L.g = lv[l].first;
            for (int a = 0; a < 3; ++a) {
                L.fac[a] = lv[l].second[a];
                L.b[a] = balloc<float>(b, L.g.nface(a), e);
            }
            L.x = l == 0 ? nullptr : balloc<float>(b, L.g.ncell(), e);
            L.f = l == 0 ? nullptr : balloc<float>(b, L.g.ncell(), e);
        }
        const int64_t N = H.g0.ncell();
        for (int a = 0; a < 3; ++a) I.b64[a] = balloc<double>(b, H.g0.nface(a), e);
        I.f64 = balloc<double>(b, N, e);
        I.r = balloc<float>(b, N, e);
        I.z = balloc<float>(b, N, e);
        I.d = balloc<float>(b, N, e);
        I.q = balloc<float>(b, N, e);
        I.e = balloc<float>(b, N, e);
        I.cinv = I.dense ? balloc<double>(b, (int64_t)I.ncoarse * I.ncoarse, e) : nullptr;
    }
    b->d_stats = balloc<double>(b, 8 * (int64_t)n, e);
    b->d_bar = balloc<unsigned>(b, 2 * (int64_t)n, e);
    b->d_err = balloc<int>(b, 1, e);
    b->d_inst = balloc<BInst>(b, n, e);
    b->d_scalars = balloc<double>(b, 3 * (int64_t)n, e);
    {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_kernel, kBT, 0);
        b->max_ctas = std::max(1, sms * per_sm);
        b->d_part = balloc<double>(b, 8 * (int64_t)b->max_ctas, e);
    }
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_stats, sizeof(double) * 8 * n);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_scalars, sizeof(double) * 3 * n);
    paris_status s = e == cudaSuccess ? PARIS_OK : PARIS_ERR_NO_MEMORY;
    if (s == PARIS_OK) s = build_descriptors(b);
    set_params(b);
    if (s != PARIS_OK) {
        paris_batch_destroy(b);
        return s;
    }
    *out = b;
    return PARIS_OK;
}

paris_status paris_batch_destroy(paris_batch* b) {
    if (!b) return PARIS_ERR_INVALID_ARG;
    cudaStreamSynchronize(b->st);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (void* p : b->allocs) cudaFree(p);
    if (b->h_stats) cudaFreeHost(b->h_stats);
    if (b->h_scalars) cudaFreeHost(b->h_scalars);
    if (b->ev) cudaEventDestroy(b->ev);
    if (b->st) cudaStreamDestroy(b->st);
    delete b;
    return PARIS_OK;
}

paris_status paris_batch_layout(const paris_batch* b, int64_t* cell_off, int64_t* xf_off,
                                int64_t* yf_off, int64_t* zf_off) {
    if (!b || !cell_off || !xf_off || !yf_off || !zf_off) return PARIS_ERR_INVALID_ARG;
    for (int i = 0; i < b->n; ++i) {
        cell_off[i] = b->hi[i].cell_off;
        xf_off[i] = b->hi[i].face_off[0];
        yf_off[i] = b->hi[i].face_off[1];
        zf_off[i] = b->hi[i].face_off[2];
    }
    cell_off[b->n] = b->cells;
    xf_off[b->n] = b->faces[0];
    yf_off[b->n] = b->faces[1];
    zf_off[b->n] = b->faces[2];
    return PARIS_OK;
}

int paris_batch_launch_ctas(const paris_batch* b) { return b ? b->grid : -1; }

}  // extern "C"

namespace {

paris_status note_error(cudaError_t e) {
    paris_internal_note_cuda_error(e);
    return PARIS_ERR_CUDA;
}

// Enqueue one batch step on the stream: scalars, barrier reset, the
// persistent launch, the stats copy (capturable).
cudaError_t enqueue_step(paris_batch* b) {
    cudaError_t e = cudaMemcpyAsync(b->d_scalars, b->h_scalars, sizeof(double) * 3 * b->n,
                                    cudaMemcpyHostToDevice, b->st);
    if (e != cudaSuccess) return e;
    batch_scalars_kernel<<<(b->n + 127) / 128, 128, 0, b->st>>>(b->n, b->d_scalars, b->d_inst);
    count_launch();
    if ((e = cudaMemsetAsync(b->d_bar, 0, sizeof(unsigned) * 2 * b->n, b->st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b->d_err, 0, sizeof(int), b->st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b->d_stats, 0, sizeof(double) * 8 * b->n, b->st)) != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->grid);
    cfg.blockDim = dim3(kBT);
    cfg.stream = b->st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const BInst* insts = b->d_inst;
    const int* cta = b->d_cta;
    BParams P = b->prm;
    int* err = b->d_err;
    e = cudaLaunchKernelEx(&cfg, persistent_kernel, insts, cta, P, err);
    count_launch();
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(b->h_stats, b->d_stats, sizeof(double) * 8 * b->n, cudaMemcpyDeviceToHost, b->st);
}

paris_status run_step(paris_batch* b, const double* C, const double* rho1, const double* rho2,
                      const double* dt, double* u, double* v, double* w, double* p, paris_stats* st,
                      bool use_graph) {
    if (!b || !C || !rho1 || !rho2 || !dt || !u || !v || !w || !p) return PARIS_ERR_INVALID_ARG;
    for (int i = 0; i < b->n; ++i) {
        if (!(rho1[i] > 0) || !(rho2[i] > 0) || !(dt[i] > 0)) return PARIS_ERR_INVALID_ARG;
        b->h_scalars[3 * i] = rho1[i];
        b->h_scalars[3 * i + 1] = rho2[i];
        b->h_scalars[3 * i + 2] = dt[i];
    }
    // order the step after the caller's pending work (e.g. filling the pools)
    if (cudaEventRecord(b->ev, b->user) != cudaSuccess || cudaStreamWaitEvent(b->st, b->ev, 0) != cudaSuccess)
        return note_error(cudaGetLastError());
    const void* key[5] = {C, u, v, w, p};
    const bool same = std::equal(key, key + 5, b->graph_key);
    if (!same) {
        // pool pointers changed: rewrite the descriptors, drop the graph
        for (int i = 0; i < b->n; ++i) {
            BInst& I = b->h_inst[i];
            const HostInst& H = b->hi[i];
            I.C = C + H.cell_off;
            I.p = p + H.cell_off;
            I.u = u + H.face_off[0];
            I.v = v + H.face_off[1];
            I.w = w + H.face_off[2];
        }
        cudaError_t e1 = cudaMemcpyAsync(b->d_inst, b->h_inst.data(), sizeof(BInst) * b->n,
                                          cudaMemcpyHostToDevice, b->st);
        if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(b->st);
        if (e1 != cudaSuccess) return note_error(e1);
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        std::copy(key, key + 5, b->graph_key);
    }
    cudaError_t e = cudaSuccess;
    if (use_graph) {
        if (!b->exec) {
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e2 = enqueue_step(b);
                e = cudaStreamEndCapture(b->st, &g);
                if (e2 != cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) return note_error(e);
        }
        e = cudaGraphLaunch(b->exec, b->st);
    } else {
        e = enqueue_step(b);
    }
    if (e != cudaSuccess) return note_error(e);
    if ((e = cudaStreamSynchronize(b->st)) != cudaSuccess) return note_error(e);
    int err = 0;
    if ((e = cudaMemcpy(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) return note_error(e);
    paris_status ret = PARIS_OK;
    for (int i = 0; i < b->n; ++i) {
        const double* s = b->h_stats + 8 * i;
        if (st) {
            st[i].iters = (int)s[0];
            st[i].outer_iters = (int)s[1];
            st[i].rel_res_l2 = s[2];
            st[i].rel_res_linf = s[3];
            st[i].mean_b_removed = 0.0;
            st[i].fell_back = 0;
            st[i].converged = (int)s[4];
            st[i].levels = (int)s[6];
        }
        if (s[5] > 0 && ret == PARIS_OK) ret = PARIS_ERR_NONFINITE;
        else if (s[4] == 0 && ret == PARIS_OK) ret = PARIS_ERR_NOT_CONVERGED;
    }
    if (err) return PARIS_ERR_TIMEOUT;
    return ret;
}

}  // namespace

extern "C" {

paris_status paris_batch_projection_step(paris_batch* b, const double* C, const double* rho1,
                                         const double* rho2, const double* dt, double* u, double* v,
                                         double* w, double* p, paris_stats* st) {
    return run_step(b, C, rho1, rho2, dt, u, v, w, p, st, true);
}

paris_status paris_batch_autotune(paris_batch* b, const double* C, const double* rho1,
                                  const double* rho2, const double* dt, const double* u,
                                  const double* v, const double* w, const char* cache_path,
                                  double* best_ms) {
    if (!b || !C || !rho1 || !rho2 || !dt || !u || !v || !w) return PARIS_ERR_INVALID_ARG;
    // cache key: device name and the instance shapes
    cudaDeviceProp prop;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    uint64_t hsh = 1469598103934665603ull;
    for (int i = 0; i < b->n; ++i)
        for (int x : {b->hi[i].grid.nx, b->hi[i].grid.ny, b->hi[i].grid.nz, b->hi[i].grid.bc[0],
                      b->hi[i].grid.bc[1], b->hi[i].grid.bc[2]})
            hsh = (hsh ^ (uint64_t)x) * 1099511628211ull;
    char key[512];
    snprintf(key, sizeof key, "%s|n=%d|shapes=%016llx|tol=%g", prop.name, b->n,
             (unsigned long long)hsh, b->opts.tol);
    if (cache_path) {
        std::ifstream in(cache_path);
        std::string line;
        while (in && std::getline(in, line)) {
            if (line.find(key) == std::string::npos) continue;
            int nu = 0, bps = 0;
            double om = 0, ms = 0;
            const char* q = strstr(line.c_str(), "\"nu\":");
            const char* r = strstr(line.c_str(), "\"omega\":");
            const char* t = strstr(line.c_str(), "\"ctas_per_sm\":");
            const char* m = strstr(line.c_str(), "\"ms\":");
            if (q && r && t && m && sscanf(q, "\"nu\":%d", &nu) == 1 && sscanf(r, "\"omega\":%lf", &om) == 1 &&
                sscanf(t, "\"ctas_per_sm\":%d", &bps) == 1 && sscanf(m, "\"ms\":%lf", &ms) == 1) {
                b->opts.nu1 = b->opts.nu2 = nu;
                b->opts.omega = om;
                if (bps != b->bps) {
                    b->bps = bps;
                    paris_status s = build_descriptors(b);
                    if (s != PARIS_OK) return s;
                    b->graph_key[0] = nullptr;  // descriptors changed
                }
                set_params(b);
                if (best_ms) *best_ms = ms;
                return PARIS_OK;
            }
        }
    }
    // scratch copies of u*, v*, w* and p for the trials (not a timed path)
    double *tu = nullptr, *tv = nullptr, *tw = nullptr, *tp = nullptr;
    if (cudaMalloc(&tu, sizeof(double) * b->faces[0]) != cudaSuccess ||
        cudaMalloc(&tv, sizeof(double) * b->faces[1]) != cudaSuccess ||
        cudaMalloc(&tw, sizeof(double) * b->faces[2]) != cudaSuccess ||
        cudaMalloc(&tp, sizeof(double) * b->cells) != cudaSuccess) {
        cudaFree(tu); cudaFree(tv); cudaFree(tw); cudaFree(tp);
        return PARIS_ERR_NO_MEMORY;
    }
    int dev_max = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&dev_max, persistent_kernel, kBT, 0);
    const int nus[3] = {1, 2, 3};
    const double oms[3] = {1.0, 1.15, 1.3};
    std::vector<int> bpss;
    for (int c : {1, 2, 4, 8})
        if (c <= dev_max) bpss.push_back(c);
    double best = INFINITY;
    int bnu = b->opts.nu1, bbps = b->bps;
    double bom = b->opts.omega;
    paris_status ret = PARIS_OK;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int bps : bpss) {
        if (sms * bps < b->n) continue;  // needs at least one CTA per instance
        b->bps = bps;
        if ((ret = build_descriptors(b)) != PARIS_OK) break;
        b->graph_key[0] = nullptr;
        for (int nu : nus)
            for (double om : oms) {
                b->opts.nu1 = b->opts.nu2 = nu;
                b->opts.omega = om;
                set_params(b);
                cudaMemcpyAsync(tu, u, sizeof(double) * b->faces[0], cudaMemcpyDeviceToDevice, b->st);
                cudaMemcpyAsync(tv, v, sizeof(double) * b->faces[1], cudaMemcpyDeviceToDevice, b->st);
                cudaMemcpyAsync(tw, w, sizeof(double) * b->faces[2], cudaMemcpyDeviceToDevice, b->st);
                cudaEventRecord(e0, b->st);
                paris_status s = run_step(b, C, rho1, rho2, dt, tu, tv, tw, tp, nullptr, false);
                cudaEventRecord(e1, b->st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (s == PARIS_OK && ms < best) {
                    best = ms;
                    bnu = nu;
                    bom = om;
                    bbps = bps;
                }
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(tu); cudaFree(tv); cudaFree(tw); cudaFree(tp);
    b->opts.nu1 = b->opts.nu2 = bnu;
    b->opts.omega = bom;
    b->bps = bbps;
    if (ret == PARIS_OK) ret = build_descriptors(b);
    b->graph_key[0] = nullptr;
    set_params(b);
    if (ret != PARIS_OK) return ret;
    if (!std::isfinite(best)) return PARIS_ERR_NOT_CONVERGED;
    if (best_ms) *best_ms = best;
    if (cache_path) {
        std::ofstream o(cache_path, std::ios::app);
        o << "{\"key\":\"" << key << "\",\"nu\":" << bnu << ",\"omega\":" << bom
          << ",\"ctas_per_sm\":" << bbps << ",\"ms\":" << best << "}\n";
    }
    return PARIS_OK;
}

paris_status paris_batch_get_tuning(const paris_batch* b, int* nu, double* omega, int* ctas_per_sm) {
    if (!b || !nu || !omega || !ctas_per_sm) return PARIS_ERR_INVALID_ARG;
    *nu = b->opts.nu1;
    *omega = b->opts.omega;
    *ctas_per_sm = b->bps;
    return PARIS_OK;
}

}  // extern "C"
