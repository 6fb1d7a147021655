// Multigrid preconditioner of the implicit viscous step (Sec. 3.2.3, Eq.
// muelliptic) and the kernels of the mixed-precision solve around it.
//
// One velocity component's SPD operator on its unknowns (the component's
// face grid without its own wall faces),
//
//     A x = sigma x - Lap_h x,      sigma = 1 / (tau nu_f),
//
// is preconditioned by an FP32 V-cycle over a hierarchy of grids coarsened
// by two along every axis together.  The kind of an axis fixes how:
//   * periodic, and the no-slip axes of a tangential component (unknowns at
//     cell centres, the wall half a cell beyond the ends, ghost value minus
//     the end value): cell-centred, m -> m/2 (m even), children 2I and 2I+1,
//     prolongation constant, restriction their average;
//   * the component's own wall axis (unknowns at faces 1 .. n-1, zero at
//     faces 0 and n): vertex-centred, m -> (m-1)/2 (m odd), coarse point J
//     at fine point 2J+1, prolongation linear, restriction full weighting
//     (1/4, 1/2, 1/4).
// The restriction is the transpose of the prolongation scaled to average, so
// the coarse equations are rediscretised at spacing 2h with the same
// boundary kinds; the coarse sigma is the restricted fine sigma.  Smoother:
// red-black Gauss-Seidel with over-relaxation where every periodic extent of
// the level is even, damped Jacobi otherwise (a periodic axis of odd length
// would give a cell two neighbours of its own colour).  The solve around it
// has the structure of the Poisson solve's mixed form: FP64 iterative
// refinement (the FP64 residual of the SPD form, the accumulation of u*)
// around an FP32 flexible CG (the V-cycle is not exactly linear: FP32,
// Gauss-Seidel) on the finest level's operator with FP32 sigma.
#include "kernels.cuh"

namespace paris {

namespace {

constexpr int kTX = 32, kTY = 8, kZ = 8;

struct HLev {
    int m[3];     // unknowns per axis
    int kind[3];  // HELM_PERIODIC / HELM_ZERO / HELM_NOSLIP
    float ih2;    // 1 / h_l^2
};

__device__ __forceinline__ int hidx(const HLev& L, int i, int j, int k) { return (k * L.m[1] + j) * L.m[0] + i; }

// the six neighbour values (or the ghost rule) and the Laplacian diagonal
// count of unknown (i, j, k): acc gets sum of neighbour values, dg the count
template <typename T, typename V>
__device__ __forceinline__ void hnb(const HLev& L, const V* __restrict__ x, int i, int j, int k, T& acc, T& dg) {
    const int pos[3] = {i, j, k};
    acc = T(0);
    dg = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int m = L.m[a];
        const int st = a == 0 ? 1 : (a == 1 ? L.m[0] : L.m[0] * L.m[1]);
        const int c = hidx(L, i, j, k);
        const int p = pos[a];
        if (L.kind[a] == HELM_PERIODIC) {
            if (m > 1) {
                acc += (T)x[p > 0 ? c - st : c + (m - 1) * st] + (T)x[p < m - 1 ? c + st : c - (m - 1) * st];
                dg += T(2);
            }
        } else {
            if (p > 0) acc += (T)x[c - st];
            if (p < m - 1) acc += (T)x[c + st];
            dg += T(2);
            if (L.kind[a] == HELM_NOSLIP) dg += T((p == 0) + (p == m - 1));  // ghost = -x_c
        }
    }
}

// one colour of red-black Gauss-Seidel (or, with JAC, a damped Jacobi sweep
// from xi into xo): x_c += omega ((f_c + acc/h^2) / (sigma_c + dg/h^2) - x_c)
template <bool JAC>
__global__ void __launch_bounds__(kTX* kTY) hmg_smooth_kernel(HLev L, const float* __restrict__ f,
                                                             const float* __restrict__ sig, const float* xi,
                                                             float* xo, int color, float omega) {
    const int i = blockIdx.x * kTX + threadIdx.x, j = blockIdx.y * kTY + threadIdx.y;
    if (i >= L.m[0] || j >= L.m[1]) return;
    const int k0 = blockIdx.z * kZ, k1 = min(k0 + kZ, L.m[2]);
    for (int k = k0; k < k1; ++k) {
        if (!JAC && ((i + j + k) & 1) != color) continue;
        const int c = hidx(L, i, j, k);
        float acc, dg;
        hnb<float>(L, xi, i, j, k, acc, dg);
        const float xc = xi[c];
        const float gs = fmaf(acc, L.ih2, f[c]) / fmaf(dg, L.ih2, sig[c]);
        xo[c] = fmaf(omega, gs - xc, xc);
    }
}

// One colour of red-black Gauss-Seidel with a thread per pair of cells
// (2t, 2t+1) of a row: the member of the pass's colour is updated, so every
// thread works on every plane of its z-segment.  Same update as the
// column kernel above.
__global__ void __launch_bounds__(kTX* kTY) hmg_rbgs_pair_kernel(HLev L, const float* __restrict__ f,
                                                                const float* __restrict__ sig, float* x, int color,
                                                                float omega) {
    pdl_wait();
    const int t = blockIdx.x * kTX + threadIdx.x, j = blockIdx.y * kTY + threadIdx.y;
    if (2 * t >= L.m[0] || j >= L.m[1]) return;
    const int k0 = blockIdx.z * kZ, k1 = min(k0 + kZ, L.m[2]);
    for (int k = k0; k < k1; ++k) {
        const int i = 2 * t + ((j + k + color) & 1);
        if (i >= L.m[0]) continue;
        const int c = hidx(L, i, j, k);
        float acc, dg;
        hnb<float>(L, x, i, j, k, acc, dg);
        const float xc = x[c];
        const float gs = fmaf(acc, L.ih2, f[c]) / fmaf(dg, L.ih2, sig[c]);
        x[c] = fmaf(omega, gs - xc, xc);
    }
}

// The same colour pass with a thread per four cells 4q .. 4q+3 of a row
// (rows of m0 % 4 == 0 cells, at least a warp's worth): every array read as
// 16-byte vectors, the two cells of the pass's colour updated, the
// x-neighbours outside the quad from the adjacent lanes (or loaded at the
// edges of the warp), the quad stored back whole (the other two cells
// unchanged: no thread writes them in this pass).  M: the updated member of
// both pairs of the quad ((j + k + color) & 1, uniform per row).
template <int M>
__device__ __forceinline__ void hrb4_row(const HLev& L, const float* __restrict__ f, const float* __restrict__ sig,
                                         float* x, float omega, int j, int k, int i0, int lane, bool act) {
    const int m0 = L.m[0], m1 = L.m[1], m2 = L.m[2], pl = m0 * m1;
    const int rowc = (k * m1 + j) * m0, c0 = rowc + i0;
    const bool py = L.kind[1] == HELM_PERIODIC, pz = L.kind[2] == HELM_PERIODIC;
    // neighbour rows and planes: present (or wrapped) and their offsets
    const bool hym = py ? m1 > 1 : j > 0, hyp = py ? m1 > 1 : j < m1 - 1;
    const bool hzm = pz ? m2 > 1 : k > 0, hzp = pz ? m2 > 1 : k < m2 - 1;
    const int oym = j > 0 ? -m0 : (m1 - 1) * m0, oyp = j < m1 - 1 ? m0 : -(m1 - 1) * m0;
    const int ozm = k > 0 ? -pl : (m2 - 1) * pl, ozp = k < m2 - 1 ? pl : -(m2 - 1) * pl;
    float X[4], F[4], S[4], YM[4] = {0.f, 0.f, 0.f, 0.f}, YP[4] = {0.f, 0.f, 0.f, 0.f},
                                ZM[4] = {0.f, 0.f, 0.f, 0.f}, ZP[4] = {0.f, 0.f, 0.f, 0.f};
    auto ld = [](float (&d)[4], const float* p) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        d[0] = v.x;
        d[1] = v.y;
        d[2] = v.z;
        d[3] = v.w;
    };
    ld(X, x + c0);
    ld(F, f + c0);
    ld(S, sig + c0);
    if (hym) ld(YM, x + c0 + oym);
    if (hyp) ld(YP, x + c0 + oyp);
    if (hzm) ld(ZM, x + c0 + ozm);
    if (hzp) ld(ZP, x + c0 + ozp);
    // x of the cells next to the quad (i0-1 and i0+4): wrapped along a periodic
    // axis, absent (0) beyond the ends of the other kinds
    const bool px = L.kind[0] == HELM_PERIODIC;
    const int il = i0 > 0 ? i0 - 1 : m0 - 1, ir = i0 + 4 < m0 ? i0 + 4 : 0;
    const bool hxl = px ? m0 > 1 : i0 > 0, hxr = px ? m0 > 1 : i0 + 4 < m0;
    const float xl_sh = __shfl_up_sync(0xffffffffu, X[3], 1), xr_sh = __shfl_down_sync(0xffffffffu, X[0], 1);
    const float xl_ld = hxl ? x[rowc + il] : 0.f, xr_ld = hxr ? x[rowc + ir] : 0.f;
    const float xl = (lane > 0 && i0 > 0) ? xl_sh : xl_ld;
    const float xr = (lane < kTX - 1 && i0 + 4 < m0) ? xr_sh : xr_ld;
    // Laplacian diagonal counts of the y and z axes (uniform per row)
    auto ends = [](int kind, int m, int p) {
        if (kind == HELM_PERIODIC) return m > 1 ? 2.f : 0.f;
        return kind == HELM_NOSLIP ? 2.f + (float)((p == 0) + (p == m - 1)) : 2.f;
    };
    const float dyz = ends(L.kind[1], m1, j) + ends(L.kind[2], m2, k);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int li = 2 * u + M, i = i0 + li;
        const float lo = li > 0 ? X[li - 1] : xl, hi = li < 3 ? X[li + 1] : xr;
        const float acc = ((lo + hi) + (YM[li] + YP[li])) + (ZM[li] + ZP[li]);
        const float dg = ends(L.kind[0], m0, i) + dyz;
        const float gs = fmaf(acc, L.ih2, F[li]) / fmaf(dg, L.ih2, S[li]);
        X[li] = fmaf(omega, gs - X[li], X[li]);
    }
    if (act) *reinterpret_cast<float4*>(x + c0) = make_float4(X[0], X[1], X[2], X[3]);
}

// (A x) of the four cells 4q .. 4q+3 of a row (the quad layout of
// hrb4_row: 16-byte vectors, x-neighbours from the adjacent lanes); X: x of
// the quad as loaded.  Same per-cell arithmetic as hmg_residual_kernel.
__device__ __forceinline__ void hop4(const HLev& L, const float* __restrict__ x, const float* __restrict__ sig,
                                     int j, int k, int i0, int lane, float (&X)[4], float (&AX)[4]) {
    const int m0 = L.m[0], m1 = L.m[1], m2 = L.m[2], pl = m0 * m1;
    const int rowc = (k * m1 + j) * m0, c0 = rowc + i0;
    const bool py = L.kind[1] == HELM_PERIODIC, pz = L.kind[2] == HELM_PERIODIC, px = L.kind[0] == HELM_PERIODIC;
    const bool hym = py ? m1 > 1 : j > 0, hyp = py ? m1 > 1 : j < m1 - 1;
    const bool hzm = pz ? m2 > 1 : k > 0, hzp = pz ? m2 > 1 : k < m2 - 1;
    const int oym = j > 0 ? -m0 : (m1 - 1) * m0, oyp = j < m1 - 1 ? m0 : -(m1 - 1) * m0;
    const int ozm = k > 0 ? -pl : (m2 - 1) * pl, ozp = k < m2 - 1 ? pl : -(m2 - 1) * pl;
    float S[4], YM[4] = {0.f, 0.f, 0.f, 0.f}, YP[4] = {0.f, 0.f, 0.f, 0.f}, ZM[4] = {0.f, 0.f, 0.f, 0.f},
                ZP[4] = {0.f, 0.f, 0.f, 0.f};
    auto ld = [](float (&d)[4], const float* p) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        d[0] = v.x;
        d[1] = v.y;
        d[2] = v.z;
        d[3] = v.w;
    };
    ld(X, x + c0);
    ld(S, sig + c0);
    if (hym) ld(YM, x + c0 + oym);
    if (hyp) ld(YP, x + c0 + oyp);
    if (hzm) ld(ZM, x + c0 + ozm);
    if (hzp) ld(ZP, x + c0 + ozp);
    const int il = i0 > 0 ? i0 - 1 : m0 - 1, ir = i0 + 4 < m0 ? i0 + 4 : 0;
    const bool hxl = px ? m0 > 1 : i0 > 0, hxr = px ? m0 > 1 : i0 + 4 < m0;
    const float xl_sh = __shfl_up_sync(0xffffffffu, X[3], 1), xr_sh = __shfl_down_sync(0xffffffffu, X[0], 1);
    const float xl_ld = hxl ? __ldg(x + rowc + il) : 0.f, xr_ld = hxr ? __ldg(x + rowc + ir) : 0.f;
    const float xl = (lane > 0 && i0 > 0) ? xl_sh : xl_ld;
    const float xr = (lane < kTX - 1 && i0 + 4 < m0) ? xr_sh : xr_ld;
    auto ends = [](int kind, int m, int p) {
        if (kind == HELM_PERIODIC) return m > 1 ? 2.f : 0.f;
        return kind == HELM_NOSLIP ? 2.f + (float)((p == 0) + (p == m - 1)) : 2.f;
    };
    const float dyz = ends(L.kind[1], m1, j) + ends(L.kind[2], m2, k);
#pragma unroll
    for (int li = 0; li < 4; ++li) {
        const float lo = li > 0 ? X[li - 1] : xl, hi = li < 3 ? X[li + 1] : xr;
        const float acc = ((lo + hi) + (YM[li] + YP[li])) + (ZM[li] + ZP[li]);
        const float dg = ends(L.kind[0], m0, i0 + li) + dyz;
        AX[li] = fmaf(dg, L.ih2, S[li]) * X[li] - acc * L.ih2;
    }
}

// r = f - A x (quads)
__global__ void __launch_bounds__(kTX* kTY) hmg_residual4_kernel(HLev L, const float* __restrict__ f,
                                                                const float* __restrict__ sig,
                                                                const float* __restrict__ x, float* __restrict__ r) {
    pdl_wait();
    const int j = blockIdx.y * kTY + threadIdx.y;
    if (j >= L.m[1]) return;
    const int k = blockIdx.z, lane = threadIdx.x;
    const int nq = L.m[0] / 4, q = blockIdx.x * kTX + lane;
    const bool act = q < nq;
    const int i0 = 4 * (act ? q : nq - 1);
    float X[4], AX[4];
    hop4(L, x, sig, j, k, i0, lane, X, AX);
    if (act) {
        const int c0 = (k * L.m[1] + j) * L.m[0] + i0;
        const float4 fv = __ldg(reinterpret_cast<const float4*>(f + c0));
        *reinterpret_cast<float4*>(r + c0) = make_float4(fv.x - AX[0], fv.y - AX[1], fv.z - AX[2], fv.w - AX[3]);
    }
}

// q = A d (quads) and the partials of d . q
__global__ void __launch_bounds__(kTX* kTY) hmg_matvec4_kernel(HLev L, const float* __restrict__ sig,
                                                              const float* __restrict__ d, float* __restrict__ q,
                                                              double* partials, FinSpec fin) {
    pdl_wait();
    const int j = blockIdx.y * kTY + threadIdx.y;
    const int tid = threadIdx.y * kTX + threadIdx.x;
    const int jc = j < L.m[1] ? j : L.m[1] - 1;  // idle rows shadow the last row (no stores)
    const int k = blockIdx.z, lane = threadIdx.x;
    const int nq = L.m[0] / 4, qq = blockIdx.x * kTX + lane;
    const bool act = qq < nq && j < L.m[1];
    const int i0 = 4 * (qq < nq ? qq : nq - 1);
    float X[4], AX[4];
    hop4(L, d, sig, jc, k, i0, lane, X, AX);
    float dq = 0.f;
    if (act) {
        const int c0 = (k * L.m[1] + jc) * L.m[0] + i0;
        *reinterpret_cast<float4*>(q + c0) = make_float4(AX[0], AX[1], AX[2], AX[3]);
#pragma unroll
        for (int li = 0; li < 4; ++li) dq = fmaf(X[li], AX[li], dq);
    }
    double accd[1] = {(double)dq};
    const int op[1] = {0};
    block_reduce_store<1>(accd, op, partials, ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x,
                          tid);
    finalize_last_block(partials, (int64_t)gridDim.x * gridDim.y * gridDim.z, fin, tid);
}

__global__ void __launch_bounds__(kTX* kTY) hmg_rb4_kernel(HLev L, const float* __restrict__ f,
                                                          const float* __restrict__ sig, float* x, int color,
                                                          float omega) {
    pdl_wait();
    const int j = blockIdx.y * kTY + threadIdx.y;
    if (j >= L.m[1]) return;  // uniform per warp
    const int k = blockIdx.z, lane = threadIdx.x;
    const int nq = L.m[0] / 4, q = blockIdx.x * kTX + lane;
    const bool act = q < nq;
    const int i0 = 4 * (act ? q : nq - 1);  // idle lanes shadow the last quad (no stores)
    if (((j + k + color) & 1) == 0)
        hrb4_row<0>(L, f, sig, x, omega, j, k, i0, lane, act);
    else
        hrb4_row<1>(L, f, sig, x, omega, j, k, i0, lane, act);
}

// r = f - A x on a level (FP32)
__global__ void __launch_bounds__(kTX* kTY) hmg_residual_kernel(HLev L, const float* __restrict__ f,
                                                               const float* __restrict__ sig,
                                                               const float* __restrict__ x, float* __restrict__ r) {
    pdl_wait();
    const int i = blockIdx.x * kTX + threadIdx.x, j = blockIdx.y * kTY + threadIdx.y;
    if (i >= L.m[0] || j >= L.m[1]) return;
    const int k0 = blockIdx.z * kZ, k1 = min(k0 + kZ, L.m[2]);
#pragma unroll 4
    for (int k = k0; k < k1; ++k) {
        const int c = hidx(L, i, j, k);
        float acc, dg;
        hnb<float>(L, x, i, j, k, acc, dg);
        const float xc = x[c];
        r[c] = f[c] - (fmaf(dg, L.ih2, sig[c]) * xc - acc * L.ih2);
    }
}

// fine points of coarse point I along an axis and their restriction weights
struct Kids {
    int n;
    int i[3];
    float w[3];
};
__device__ __forceinline__ Kids kids(int kind, int I) {
    Kids q;
    if (kind == HELM_ZERO) {  // vertex-centred: fine 2I, 2I+1, 2I+2 (1/4, 1/2, 1/4)
        q.n = 3;
        q.i[0] = 2 * I;
        q.i[1] = 2 * I + 1;
        q.i[2] = 2 * I + 2;
        q.w[0] = 0.25f;
        q.w[1] = 0.5f;
        q.w[2] = 0.25f;
    } else {  // cell-centred: fine 2I, 2I+1 (1/2, 1/2)
        q.n = 2;
        q.i[0] = 2 * I;
        q.i[1] = 2 * I + 1;
        q.i[2] = 0;
        q.w[0] = q.w[1] = 0.5f;
        q.w[2] = 0.f;
    }
    return q;
}

// coarse = R fine (tensor product of the per-axis weights)
__global__ void __launch_bounds__(kTX* kTY) hmg_restrict_kernel(HLev F, HLev Cg, const float* __restrict__ fine,
                                                               float* __restrict__ coarse) {
    pdl_wait();
    const int I = blockIdx.x * kTX + threadIdx.x, J = blockIdx.y * kTY + threadIdx.y, K = blockIdx.z;
    if (I >= Cg.m[0] || J >= Cg.m[1]) return;
    const Kids a = kids(F.kind[0], I), b = kids(F.kind[1], J), c = kids(F.kind[2], K);
    float s = 0.f;
    for (int z = 0; z < c.n; ++z)
        for (int y = 0; y < b.n; ++y) {
            float sx = 0.f;
            for (int x = 0; x < a.n; ++x) sx = fmaf(a.w[x], fine[hidx(F, a.i[x], b.i[y], c.i[z])], sx);
            s = fmaf(c.w[z] * b.w[y], sx, s);
        }
    coarse[hidx(Cg, I, J, K)] = s;
}

// coarse points of fine point i along an axis and the prolongation weights
struct Pars {
    int n;
    int I[2];
    float w[2];
};
__device__ __forceinline__ Pars parents(int kind, int i, int mc) {
    Pars q;
    q.n = 0;
    if (kind == HELM_ZERO) {
        // fine unknown i sits at face i+1; coarse unknown J at face 2(J+1)
        const int F = i + 1;
        if ((F & 1) == 0) {
            q.n = 1;
            q.I[0] = F / 2 - 1;
            q.w[0] = 1.f;
        } else {
            const int J1 = (F - 1) / 2 - 1, J2 = (F + 1) / 2 - 1;
            if (J1 >= 0) { q.I[q.n] = J1; q.w[q.n] = 0.5f; ++q.n; }
            if (J2 < mc) { q.I[q.n] = J2; q.w[q.n] = 0.5f; ++q.n; }
        }
    } else {
        q.n = 1;
        q.I[0] = i / 2;
        q.w[0] = 1.f;
    }
    return q;
}

// x += P e (tensor product)
__global__ void __launch_bounds__(kTX* kTY) hmg_prolong_kernel(HLev F, HLev Cg, const float* __restrict__ e,
                                                              float* __restrict__ x) {
    pdl_wait();
    const int i = blockIdx.x * kTX + threadIdx.x, j = blockIdx.y * kTY + threadIdx.y, k = blockIdx.z;
    if (i >= F.m[0] || j >= F.m[1]) return;
    const Pars a = parents(F.kind[0], i, Cg.m[0]), b = parents(F.kind[1], j, Cg.m[1]),
               c = parents(F.kind[2], k, Cg.m[2]);
    float s = 0.f;
    for (int z = 0; z < c.n; ++z)
        for (int y = 0; y < b.n; ++y)
            for (int q = 0; q < a.n; ++q) s = fmaf(a.w[q] * b.w[y] * c.w[z], e[hidx(Cg, a.I[q], b.I[y], c.I[z])], s);
    x[hidx(F, i, j, k)] += s;
}

// ---------------------------------------------------------------- FP64 side

// sigma = 1/(tau nu) on the unknowns (FP64 and FP32 copies); the right-hand
// side norms of b = sigma u^n (partials |b|^2, max |b|, non-finite count, 0;
// a nu that is not > 0 counts as non-finite); u* = u^n on the unknowns
__global__ void __launch_bounds__(kTX* kTY) hmg_setup_kernel(HelmGeo g, const double* __restrict__ un,
                                                            const double* __restrict__ nu, double tau,
                                                            double* __restrict__ sig64, float* __restrict__ sig32,
                                                            double* __restrict__ us, double* partials, FinSpec fin) {
    const int i = blockIdx.x * kTX + threadIdx.x, j = blockIdx.y * kTY + threadIdx.y;
    const int tid = threadIdx.y * kTX + threadIdx.x;
    double l2 = 0.0;
    unsigned long long bk = 0;
    unsigned nf = 0;
    if (i < g.m[0] && j < g.m[1]) {
        const int k0 = blockIdx.z * kZ, k1 = min(k0 + kZ, g.m[2]);
        for (int k = k0; k < k1; ++k) {
            const int64_t p = ((int64_t)k * g.m[1] + j) * g.m[0] + i;
            const int64_t f = g.off + i + (int64_t)g.e[0] * (j + (int64_t)g.e[1] * k);
            const double nv = nu[f], v = un[f];
            const double s = 1.0 / (tau * nv);
            sig64[p] = s;
            sig32[p] = (float)s;
            us[f] = v;
            const double b = s * v;
            l2 = fma(b, b, l2);
            const unsigned long long kb = abs_key(b);
            bk = kb > bk ? kb : bk;
            nf += (key_nonfinite(kb) || !(nv > 0.0)) ? 1u : 0u;
        }
    }
    block_reduce_skc<double>(l2, bk, nf, partials, ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x,
                             tid);
    finalize_last_block(partials, (int64_t)gridDim.x * gridDim.y * gridDim.z, fin, tid);
}

// the component's wall faces of its own axis: u* = 0 there
__global__ void hmg_wall_zero_kernel(HelmGeo g, double* __restrict__ us) {
    const int c = g.comp, a1 = c == 0 ? 1 : 0, a2 = c == 2 ? 1 : 2;
    const int64_t plane = (int64_t)g.e[a1] * g.e[a2];
    const int64_t se[3] = {1, g.e[0], (int64_t)g.e[0] * g.e[1]};
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < 2 * plane; w += (int64_t)gridDim.x * blockDim.x) {
        const int side = w >= plane;
        const int64_t rem = w - side * plane;
        const int64_t i2 = rem / g.e[a1], i1 = rem - i2 * g.e[a1];
        us[i1 * se[a1] + i2 * se[a2] + (int64_t)side * (g.e[c] - 1) * se[c]] = 0.0;
    }
}

// FP64 operator on the unknowns of x stored with strides st (the face array
// of u*, or a Krylov vector): returns sigma x_c - Lap_h x at (i, j, k)
__device__ __forceinline__ double hop64(const HelmGeo& g, const double* __restrict__ x, int64_t c,
                                        const int64_t (&st)[3], int i, int j, int k, double sig) {
    const int pos[3] = {i, j, k};
    const double xc = x[c];
    double acc = 0.0, dg = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int m = g.m[a], p = pos[a];
        if (g.kind[a] == HELM_PERIODIC) {
            if (m > 1) {
                acc += x[p > 0 ? c - st[a] : c + (int64_t)(m - 1) * st[a]] +
                       x[p < m - 1 ? c + st[a] : c - (int64_t)(m - 1) * st[a]];
                dg += 2.0;
            }
        } else {
            if (p > 0) acc += x[c - st[a]];
            if (p < m - 1) acc += x[c + st[a]];
            dg += 2.0;
            if (g.kind[a] == HELM_NOSLIP) dg += (double)((p == 0) + (p == m - 1));
        }
    }
    return fma(dg, g.ih2, sig) * xc - acc * g.ih2;
}

// r = sigma u^n - A u* (u* the face array), f32 = (float) r; partials (|r|^2,
// max |r|, non-finite count)
__global__ void __launch_bounds__(kTX* kTY) hmg_residual64_kernel(HelmGeo g, const double* __restrict__ un,
                                                                 const double* __restrict__ sig,
                                                                 const double* __restrict__ us,
                                                                 double* __restrict__ r, double* partials,
                                                                 FinSpec fin) {
    pdl_wait();
    const int i = blockIdx.x * kTX + threadIdx.x, j = blockIdx.y * kTY + threadIdx.y;
    const int tid = threadIdx.y * kTX + threadIdx.x;
    double l2 = 0.0;
    unsigned long long rk = 0;
    unsigned nf = 0;
    const int64_t se[3] = {1, g.e[0], (int64_t)g.e[0] * g.e[1]};
    if (i < g.m[0] && j < g.m[1]) {
        const int k0 = blockIdx.z * kZ, k1 = min(k0 + kZ, g.m[2]);
        for (int k = k0; k < k1; ++k) {
            const int64_t p = ((int64_t)k * g.m[1] + j) * g.m[0] + i;
            const int64_t f = g.off + i + (int64_t)g.e[0] * (j + (int64_t)g.e[1] * k);
            const double s = sig[p];
            const double rp = s * un[f] - hop64(g, us, f, se, i, j, k, s);
            r[p] = rp;
            l2 = fma(rp, rp, l2);
            const unsigned long long kr = abs_key(rp);
            rk = kr > rk ? kr : rk;
            nf += key_nonfinite(kr);
        }
    }
    block_reduce_skc<double>(l2, rk, nf, partials, ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x,
                             tid);
    finalize_last_block(partials, (int64_t)gridDim.x * gridDim.y * gridDim.z, fin, tid);
}

// FP32 inner iteration: q = A d on the finest level (FP32 sigma) and the
// partials of d . q
__global__ void __launch_bounds__(kTX* kTY) hmg_matvec32_kernel(HLev L, const float* __restrict__ sig,
                                                               const float* __restrict__ d, float* __restrict__ q,
                                                               double* partials, FinSpec fin) {
    pdl_wait();
    const int i = blockIdx.x * kTX + threadIdx.x, j = blockIdx.y * kTY + threadIdx.y;
    const int tid = threadIdx.y * kTX + threadIdx.x;
    float dq = 0.f;
    if (i < L.m[0] && j < L.m[1]) {
        const int k0 = blockIdx.z * kZ, k1 = min(k0 + kZ, L.m[2]);
#pragma unroll 4
        for (int k = k0; k < k1; ++k) {
            const int c = hidx(L, i, j, k);
            float acc, dg;
            hnb<float>(L, d, i, j, k, acc, dg);
            const float dc = d[c];
            const float qc = fmaf(dg, L.ih2, sig[c]) * dc - acc * L.ih2;
            q[c] = qc;
            dq = fmaf(dc, qc, dq);
        }
    }
    double accd[1] = {(double)dq};
    const int op[1] = {0};
    block_reduce_store<1>(accd, op, partials, ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x,
                          tid);
    finalize_last_block(partials, (int64_t)gridDim.x * gridDim.y * gridDim.z, fin, tid);
}

// r32 = scale r64 (scale a power of two from the context's scalar block,
// kept until the correction is accumulated); partials of |r32|^2, max |r32|
__global__ void hmg_scale_d2f_kernel(int64_t n, const double* __restrict__ r, const Scal* __restrict__ s,
                                     float* __restrict__ r32, double* partials, FinSpec fin) {
    pdl_wait();
    const double sc = s->scale;
    float l2 = 0.f, mx = 0.f;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const float v = (float)(sc * r[c]);
        r32[c] = v;
        l2 = fmaf(v, v, l2);
        mx = fmaxf(mx, fabsf(v));
    }
    double acc[2] = {(double)l2, (double)mx};
    const int op[2] = {0, 1};
    block_reduce_store<2>(acc, op, partials, blockIdx.x, threadIdx.x);
    finalize_last_block(partials, gridDim.x, fin, threadIdx.x);
}

// u* += e / scale on the unknowns of the face array
__global__ void __launch_bounds__(kTX* kTY) hmg_accumulate_kernel(HelmGeo g, const float* __restrict__ e,
                                                                 const Scal* __restrict__ s, double* __restrict__ us) {
    pdl_wait();
    const int i = blockIdx.x * kTX + threadIdx.x, j = blockIdx.y * kTY + threadIdx.y;
    if (i >= g.m[0] || j >= g.m[1]) return;
    const double inv = s->inv_scale;
    const int k0 = blockIdx.z * kZ, k1 = min(k0 + kZ, g.m[2]);
    for (int k = k0; k < k1; ++k) {
        const int64_t p = ((int64_t)k * g.m[1] + j) * g.m[0] + i;
        const int64_t f = g.off + i + (int64_t)g.e[0] * (j + (int64_t)g.e[1] * k);
        us[f] = fma((double)e[p], inv, us[f]);
    }
}

inline dim3 hgrid(const int (&m)[3], int zper) {
    return dim3((m[0] + kTX - 1) / kTX, (m[1] + kTY - 1) / kTY, (m[2] + zper - 1) / zper);
}

}  // namespace

// ------------------------------------------------------------------ plan

HelmPlan helm_plan(const HelmGeo& g, int max_levels) {
    HelmPlan P{};
    int m[3] = {g.m[0], g.m[1], g.m[2]};
    double h2 = 1.0 / g.ih2;
    for (int l = 0; l < max_levels && l < kHelmMaxLevels; ++l) {
        for (int a = 0; a < 3; ++a) {
            P.lv[l].m[a] = m[a];
            P.lv[l].kind[a] = g.kind[a];
        }
        P.lv[l].ih2 = 1.0 / h2;
        P.nl = l + 1;
        bool ok = true;
        int mc[3];
        for (int a = 0; a < 3; ++a) {
            if (g.kind[a] == HELM_ZERO) {
                ok = ok && (m[a] % 2 == 1) && m[a] >= 5;
                mc[a] = (m[a] - 1) / 2;
            } else {
                ok = ok && (m[a] % 2 == 0) && m[a] >= 4;
                mc[a] = m[a] / 2;
            }
        }
        if (!ok) break;
        for (int a = 0; a < 3; ++a) m[a] = mc[a];
        h2 *= 4.0;
    }
    return P;
}

// ------------------------------------------------------------- launchers

namespace {
inline HLev hlev(const HelmLevelDesc& d) {
    HLev L;
    for (int a = 0; a < 3; ++a) {
        L.m[a] = d.m[a];
        L.kind[a] = d.kind[a];
    }
    L.ih2 = (float)d.ih2;
    return L;
}
inline int64_t hcount(const HelmLevelDesc& d) { return (int64_t)d.m[0] * d.m[1] * d.m[2]; }
inline bool rb_ok(const HelmLevelDesc& d) {
    for (int a = 0; a < 3; ++a)
        if (d.kind[a] == HELM_PERIODIC && d.m[a] % 2 == 1 && d.m[a] > 1) return false;
    return true;
}
}  // namespace

int64_t launch_hmg_setup(const HelmGeo& g, const double* un, const double* nu, double tau, double* sig64,
                         float* sig32, double* us, double* partials, cudaStream_t st, FinSpec fin) {
    const dim3 gr = hgrid(g.m, kZ);
    hmg_setup_kernel<<<gr, dim3(kTX, kTY), 0, st>>>(g, un, nu, tau, sig64, sig32, us, partials, fin);
    count_launch();
    if (g.wall) {
        const int c = g.comp, a1 = c == 0 ? 1 : 0, a2 = c == 2 ? 1 : 2;
        const int64_t n = 2 * (int64_t)g.e[a1] * g.e[a2];
        hmg_wall_zero_kernel<<<elementwise_blocks(n), kRedThreads, 0, st>>>(g, us);
        count_launch();
    }
    return (int64_t)gr.x * gr.y * gr.z;
}

void launch_hmg_sigma(const HelmPlan& P, float* const* sig, cudaStream_t st) {
    for (int l = 0; l + 1 < P.nl; ++l) {
        const HLev F = hlev(P.lv[l]), Cg = hlev(P.lv[l + 1]);
        dim3 gr((Cg.m[0] + kTX - 1) / kTX, (Cg.m[1] + kTY - 1) / kTY, Cg.m[2]);
        launch_pdl(hmg_restrict_kernel, gr, dim3(kTX, kTY), 0, st, F, Cg, sig[l], sig[l + 1]);
        count_launch();
    }
}

int64_t launch_hmg_residual64(const HelmGeo& g, const double* un, const double* sig, const double* us, double* r,
                              double* partials, cudaStream_t st, FinSpec fin) {
    const dim3 gr = hgrid(g.m, kZ);
    launch_pdl(hmg_residual64_kernel, gr, dim3(kTX, kTY), 0, st, g, un, sig, us, r, partials, fin);
    count_launch();
    return (int64_t)gr.x * gr.y * gr.z;
}

// z32 = V f32 on FP32 vectors of the finest level (f32 and z32 are not
// the work arrays of level 0, which the V-cycle uses for its own x and f)
static void hmg_vcycle_core(const HelmPlan& P, const HelmWork& W, const float* f0, float* x0, int nu1, int nu2,
                            int coarse_sweeps, float omega, cudaStream_t st);

void launch_hmg_vcycle32(const HelmPlan& P, const HelmWork& W, const float* r32, float* z32, int nu1, int nu2,
                         int coarse_sweeps, float omega, cudaStream_t st) {
    hmg_vcycle_core(P, W, r32, z32, nu1, nu2, coarse_sweeps, omega, st);
}

static void hmg_vcycle_core(const HelmPlan& P, const HelmWork& W, const float* f0, float* x0, int nu1, int nu2,
                            int coarse_sweeps, float omega, cudaStream_t st) {
    auto F = [&](int l) { return l == 0 ? f0 : (const float*)W.f[l]; };
    auto X = [&](int l) { return l == 0 ? x0 : W.x[l]; };
    auto smooth = [&](int l, int sweeps, bool reverse) {
        const HLev L = hlev(P.lv[l]);
        const dim3 gr = hgrid(P.lv[l].m, kZ);
        const bool quads = P.lv[l].m[0] % 4 == 0 && P.lv[l].m[0] >= 4 * kTX &&
                           ((uintptr_t)F(l) | (uintptr_t)W.sig[l] | (uintptr_t)X(l)) % 16 == 0;
        if (rb_ok(P.lv[l]) && quads) {
            const dim3 g4((P.lv[l].m[0] / 4 + kTX - 1) / kTX, (P.lv[l].m[1] + kTY - 1) / kTY, P.lv[l].m[2]);
            for (int s = 0; s < sweeps; ++s)
                for (int h = 0; h < 2; ++h) {
                    const int color = reverse ? 1 - h : h;
                    launch_pdl(hmg_rb4_kernel, g4, dim3(kTX, kTY), 0, st, L, F(l), W.sig[l], X(l), color,
                        omega);
                    count_launch();
                }
        } else if (rb_ok(P.lv[l])) {
            const dim3 gp(((P.lv[l].m[0] + 1) / 2 + kTX - 1) / kTX, gr.y, gr.z);
            for (int s = 0; s < sweeps; ++s)
                for (int h = 0; h < 2; ++h) {
                    const int color = reverse ? 1 - h : h;
                    launch_pdl(hmg_rbgs_pair_kernel, gp, dim3(kTX, kTY), 0, st, L, F(l), W.sig[l], X(l), color,
                        omega);
                    count_launch();
                }
        } else {  // damped Jacobi, ping-pong through the level's residual buffer, ending in x
            const int64_t n = hcount(P.lv[l]);
            for (int s = 0; s < sweeps; ++s) {
                hmg_smooth_kernel<true><<<gr, dim3(kTX, kTY), 0, st>>>(L, F(l), W.sig[l], X(l), W.r[l], 0,
                                                                      0.8f);
                cudaMemcpyAsync(X(l), W.r[l], sizeof(float) * n, cudaMemcpyDeviceToDevice, st);
                count_launch();
            }
        }
    };
    for (int l = 0; l < P.nl; ++l) {
        cudaMemsetAsync(X(l), 0, sizeof(float) * hcount(P.lv[l]), st);
        if (l == P.nl - 1) {
            smooth(l, coarse_sweeps, false);
            break;
        }
        smooth(l, nu1, false);
        const HLev L = hlev(P.lv[l]), Cg = hlev(P.lv[l + 1]);
        const bool q4 = P.lv[l].m[0] % 4 == 0 && P.lv[l].m[0] >= 4 * kTX &&
                        ((uintptr_t)F(l) | (uintptr_t)W.sig[l] | (uintptr_t)X(l) | (uintptr_t)W.r[l]) % 16 == 0;
        if (q4)
            launch_pdl(hmg_residual4_kernel,
                       dim3((P.lv[l].m[0] / 4 + kTX - 1) / kTX, (P.lv[l].m[1] + kTY - 1) / kTY, P.lv[l].m[2]),
                       dim3(kTX, kTY), 0, st, L, F(l), W.sig[l], X(l), W.r[l]);
        else
            launch_pdl(hmg_residual_kernel, hgrid(P.lv[l].m, kZ), dim3(kTX, kTY), 0, st, L, F(l), W.sig[l],
                X(l), W.r[l]);
        dim3 gr((Cg.m[0] + kTX - 1) / kTX, (Cg.m[1] + kTY - 1) / kTY, Cg.m[2]);
        launch_pdl(hmg_restrict_kernel, gr, dim3(kTX, kTY), 0, st, L, Cg, W.r[l], W.f[l + 1]);
        count_launch(2);
    }
    for (int l = P.nl - 2; l >= 0; --l) {
        const HLev L = hlev(P.lv[l]), Cg = hlev(P.lv[l + 1]);
        dim3 gr((L.m[0] + kTX - 1) / kTX, (L.m[1] + kTY - 1) / kTY, L.m[2]);
        launch_pdl(hmg_prolong_kernel, gr, dim3(kTX, kTY), 0, st, L, Cg, X(l + 1), X(l));
        count_launch();
        smooth(l, nu2, true);
    }
}

int64_t helm_max_blocks(const HelmGeo& g) {
    const dim3 gr = hgrid(g.m, kZ);
    return (int64_t)gr.x * gr.y * gr.z;
}

}  // namespace paris

namespace paris {

int64_t launch_hmg_matvec32(const HelmPlan& P, const float* sig, const float* d, float* q, double* partials,
                            cudaStream_t st, FinSpec fin) {
    const HLev L = hlev(P.lv[0]);
    // quads where the rows fill a warp; one partial per block, within the
    // context's partial slots (four per block of the z-loop grid)
    const int64_t blocks4 = (int64_t)((L.m[0] / 4 + kTX - 1) / kTX) * ((L.m[1] + kTY - 1) / kTY) * L.m[2];
    const dim3 gz = hgrid(P.lv[0].m, kZ);
    if (L.m[0] % 4 == 0 && L.m[0] >= 4 * kTX && ((uintptr_t)sig | (uintptr_t)d | (uintptr_t)q) % 16 == 0 &&
        blocks4 <= 4 * (int64_t)gz.x * gz.y * gz.z) {
        const dim3 g4((L.m[0] / 4 + kTX - 1) / kTX, (L.m[1] + kTY - 1) / kTY, L.m[2]);
        launch_pdl(hmg_matvec4_kernel, g4, dim3(kTX, kTY), 0, st, L, sig, d, q, partials, fin);
        count_launch();
        return blocks4;
    }
    const dim3 gr = hgrid(P.lv[0].m, kZ);
    launch_pdl(hmg_matvec32_kernel, gr, dim3(kTX, kTY), 0, st, L, sig, d, q, partials, fin);
    count_launch();
    return (int64_t)gr.x * gr.y * gr.z;
}

int64_t launch_hmg_scale_d2f(int64_t n, const double* r, const Scal* s, float* r32, double* partials,
                             cudaStream_t st, FinSpec fin) {
    const int nb = elementwise_blocks(n);
    launch_pdl(hmg_scale_d2f_kernel, nb, kRedThreads, 0, st, n, r, s, r32, partials, fin);
    count_launch();
    return nb;
}

void launch_hmg_accumulate(const HelmGeo& g, const float* e, const Scal* s, double* us, cudaStream_t st) {
    launch_pdl(hmg_accumulate_kernel, hgrid(g.m, kZ), dim3(kTX, kTY), 0, st, g, e, s, us);
    count_launch();
}

}  // namespace paris
