// Implicit viscous step on one velocity component (Sec. 3.2.3, Eq.
// muelliptic): the kernels of the Jacobi-preconditioned conjugate gradients
// that solve its symmetric positive definite form
//
//     (diag(1/(tau nu)) - Lap_h) u* = u^n / (tau nu)
//
// on the component's unknowns, its face grid without the wall faces of its
// own axis (where the component is zero).  Lap_h is the 7-point Laplacian
// with spacing h; beyond the ends of an axis the value is the wrapped one
// (periodic), zero (the component's own wall faces) or minus the end value
// (no-slip for a tangential component: zero velocity on the wall, half a
// cell away, Sec. 2.2).
//
// u^n, nu and u* are full face arrays (the library's face layout); the
// Krylov vectors r, z, d, q hold only the unknowns, x fastest.  The Jacobi
// step z = r / diag is fused into the kernels that produce r, which also
// reduce r . r, max |r|, the non-finite count and r . z.
#include "kernels.cuh"

namespace paris {

namespace {

__device__ __forceinline__ void helm_pos(const HelmGeo& g, int64_t p, int (&pos)[3]) {
    const int64_t t = p / g.m[0];
    pos[0] = (int)(p - t * g.m[0]);
    pos[1] = (int)(t % g.m[1]);
    pos[2] = (int)(t / g.m[1]);
}

// index in the full face array of the unknown at pos
__device__ __forceinline__ int64_t helm_face(const HelmGeo& g, const int (&pos)[3]) {
    return g.off + pos[0] + (int64_t)g.e[0] * (pos[1] + (int64_t)g.e[1] * pos[2]);
}

// Lap_h x at the entry c of x (position pos, value xc); st: strides of x
__device__ __forceinline__ double helm_lap(const HelmGeo& g, const double* __restrict__ x, int64_t c,
                                           const int64_t (&st)[3], const int (&pos)[3], double xc) {
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int m = g.m[a];
        const int kind = g.kind[a];
        const double end = kind == HELM_ZERO ? 0.0 : -xc;  // beyond a wall
        const double lo = pos[a] > 0 ? x[c - st[a]] : (kind == HELM_PERIODIC ? x[c + (int64_t)(m - 1) * st[a]] : end);
        const double hi = pos[a] < m - 1 ? x[c + st[a]] : (kind == HELM_PERIODIC ? x[c - (int64_t)(m - 1) * st[a]] : end);
        s += (lo + hi) - 2.0 * xc;
    }
    return s * g.ih2;
}

// diagonal of diag(1/(tau nu)) - Lap_h at pos
__device__ __forceinline__ double helm_diag(const HelmGeo& g, const int (&pos)[3], double inv_tnu) {
    double d = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int m = g.m[a];
        if (g.kind[a] == HELM_PERIODIC) {
            d += m > 1 ? 2.0 : 0.0;  // one point along a periodic axis is its own neighbour
        } else {
            d += 2.0;
            if (g.kind[a] == HELM_NOSLIP) d += (pos[a] == 0 ? 1.0 : 0.0) + (pos[a] == m - 1 ? 1.0 : 0.0);
        }
    }
    return inv_tnu + d * g.ih2;
}

// u* = u^n on the unknowns (the initial guess), 0 on the component's wall
// faces; partials of |b|^2, max |b|, the non-finite count (a nu that is not
// positive counts) and 0, with b = u^n / (tau nu)
__global__ void helm_init_kernel(HelmGeo g, int64_t n, const double* __restrict__ un,
                                 const double* __restrict__ nu, double tau, double* __restrict__ us,
                                 double* partials, FinSpec fin) {
    double l2 = 0.0, mx = 0.0;
    unsigned nf = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t p = t0; p < n; p += stride) {
        int pos[3];
        helm_pos(g, p, pos);
        const int64_t f = helm_face(g, pos);
        const double v = un[f];
        const double nv = nu[f];
        us[f] = v;
        const double b = v / (tau * nv);
        l2 = fma(b, b, l2);
        mx = fmax(mx, fabs(b));
        nf += (isfinite(b) && nv > 0.0) ? 0u : 1u;
    }
    // the two wall planes of the component's own axis (none along a periodic axis)
    if (g.wall) {
        const int c = g.comp, a1 = c == 0 ? 1 : 0, a2 = c == 2 ? 1 : 2;
        const int64_t plane = (int64_t)g.e[a1] * g.e[a2];
        const int64_t se[3] = {1, g.e[0], (int64_t)g.e[0] * g.e[1]};
        for (int64_t w = t0; w < 2 * plane; w += stride) {
            const int side = w >= plane;
            const int64_t rem = w - side * plane;
            const int64_t i2 = rem / g.e[a1];
            const int64_t i1 = rem - i2 * g.e[a1];
            us[i1 * se[a1] + i2 * se[a2] + (int64_t)side * (g.e[c] - 1) * se[c]] = 0.0;
        }
    }
    double acc[4] = {l2, mx, (double)nf, 0.0};
    const int op[4] = {0, 1, 0, 1};
    block_reduce_store<4>(acc, op, partials, blockIdx.x, threadIdx.x);
    finalize_last_block(partials, gridDim.x, fin, threadIdx.x);
}

// r = u^n/(tau nu) - (x/(tau nu) - Lap_h x), z = r / diag; partials of
// r . r, max |r|, the non-finite count, r . z
__global__ void helm_residual_kernel(HelmGeo g, int64_t n, const double* __restrict__ un,
                                     const double* __restrict__ nu, double tau, const double* __restrict__ x,
                                     double* __restrict__ r, double* __restrict__ z, double* partials,
                                     FinSpec fin) {
    double l2 = 0.0, mx = 0.0, rz = 0.0;
    unsigned nf = 0;
    const int64_t se[3] = {1, g.e[0], (int64_t)g.e[0] * g.e[1]};
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        int pos[3];
        helm_pos(g, p, pos);
        const int64_t f = helm_face(g, pos);
        const double xc = x[f];
        const double inv_tnu = 1.0 / (tau * nu[f]);
        const double rp = (un[f] - xc) * inv_tnu + helm_lap(g, x, f, se, pos, xc);
        const double zp = rp / helm_diag(g, pos, inv_tnu);
        r[p] = rp;
        z[p] = zp;
        l2 = fma(rp, rp, l2);
        mx = fmax(mx, fabs(rp));
        rz = fma(rp, zp, rz);
        nf += isfinite(rp) ? 0u : 1u;
    }
    double acc[4] = {l2, mx, (double)nf, rz};
    const int op[4] = {0, 1, 0, 0};
    block_reduce_store<4>(acc, op, partials, blockIdx.x, threadIdx.x);
    finalize_last_block(partials, gridDim.x, fin, threadIdx.x);
}

// q = d/(tau nu) - Lap_h d and the partials of d . q
__global__ void helm_matvec_dot_kernel(HelmGeo g, int64_t n, const double* __restrict__ nu, double tau,
                                       const double* __restrict__ d, double* __restrict__ q, double* partials,
                                       FinSpec fin) {
    double dq = 0.0;
    const int64_t su[3] = {1, g.m[0], (int64_t)g.m[0] * g.m[1]};
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        int pos[3];
        helm_pos(g, p, pos);
        const double dc = d[p];
        const double qp = dc / (tau * nu[helm_face(g, pos)]) - helm_lap(g, d, p, su, pos, dc);
        q[p] = qp;
        dq = fma(dc, qp, dq);
    }
    double acc[1] = {dq};
    const int op[1] = {0};
    block_reduce_store<1>(acc, op, partials, blockIdx.x, threadIdx.x);
    finalize_last_block(partials, gridDim.x, fin, threadIdx.x);
}

// x += alpha d, r -= alpha q, z = r / diag; partials as the residual kernel's
__global__ void helm_update_kernel(HelmGeo g, int64_t n, const double* __restrict__ nu, double tau,
                                   const Scal* __restrict__ s, const double* __restrict__ d,
                                   const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r,
                                   double* __restrict__ z, double* partials, FinSpec fin) {
    const double alpha = s->alpha;
    double l2 = 0.0, mx = 0.0, rz = 0.0;
    unsigned nf = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        int pos[3];
        helm_pos(g, p, pos);
        const int64_t f = helm_face(g, pos);
        x[f] = fma(alpha, d[p], x[f]);
        const double rp = fma(-alpha, q[p], r[p]);
        const double zp = rp / helm_diag(g, pos, 1.0 / (tau * nu[f]));
        r[p] = rp;
        z[p] = zp;
        l2 = fma(rp, rp, l2);
        mx = fmax(mx, fabs(rp));
        rz = fma(rp, zp, rz);
        nf += isfinite(rp) ? 0u : 1u;
    }
    double acc[4] = {l2, mx, (double)nf, rz};
    const int op[4] = {0, 1, 0, 0};
    block_reduce_store<4>(acc, op, partials, blockIdx.x, threadIdx.x);
    finalize_last_block(partials, gridDim.x, fin, threadIdx.x);
}

// nu_f = (mu_L + mu_R) / (rho_L + rho_R) on every face of the component,
// mu and rho from Eq. muH in the two cells sharing the face; 0 on its wall
// faces.  Rounded products and sums (no contraction), in the order written.
__global__ void helm_face_nu_kernel(HelmGeo g, int64_t nfull, int nx, int ny, const double* __restrict__ C,
                                    double mu1, double mu2, double rho1, double rho2, double* __restrict__ nu) {
    const int c = g.comp;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nfull; f += (int64_t)gridDim.x * blockDim.x) {
        int pos[3];
        const int64_t t = f / g.e[0];
        pos[0] = (int)(f - t * g.e[0]);
        pos[1] = (int)(t % g.e[1]);
        pos[2] = (int)(t / g.e[1]);
        if (g.wall && (pos[c] == 0 || pos[c] == g.e[c] - 1)) {
            nu[f] = 0.0;
            continue;
        }
        // face pos[c] lies between cells pos[c]-1 (wrapped along a periodic axis) and pos[c]
        int lo[3] = {pos[0], pos[1], pos[2]};
        lo[c] = pos[c] > 0 ? pos[c] - 1 : g.e[c] - 1;
        const double cl = C[((int64_t)lo[2] * ny + lo[1]) * nx + lo[0]];
        const double cr = C[((int64_t)pos[2] * ny + pos[1]) * nx + pos[0]];
        const double mul = __dadd_rn(__dmul_rn(mu1, cl), __dmul_rn(mu2, __dsub_rn(1.0, cl)));
        const double mur = __dadd_rn(__dmul_rn(mu1, cr), __dmul_rn(mu2, __dsub_rn(1.0, cr)));
        const double rhol = __dadd_rn(__dmul_rn(rho1, cl), __dmul_rn(rho2, __dsub_rn(1.0, cl)));
        const double rhor = __dadd_rn(__dmul_rn(rho1, cr), __dmul_rn(rho2, __dsub_rn(1.0, cr)));
        nu[f] = __dadd_rn(mul, mur) / __dadd_rn(rhol, rhor);
    }
}

}  // namespace

HelmGeo helm_geo(const Geo& g0, int comp, double h) {
    HelmGeo g{};
    const int n[3] = {g0.nx, g0.ny, g0.nz};
    const int wl[3] = {g0.wx, g0.wy, g0.wz};
    g.comp = comp;
    g.wall = wl[comp] ? 1 : 0;
    for (int a = 0; a < 3; ++a) {
        g.e[a] = n[a] + (a == comp && wl[a] ? 1 : 0);
        g.m[a] = n[a] - (a == comp && wl[a] ? 1 : 0);
        g.kind[a] = !wl[a] ? HELM_PERIODIC : (a == comp ? HELM_ZERO : HELM_NOSLIP);
    }
    const int64_t se[3] = {1, g.e[0], (int64_t)g.e[0] * g.e[1]};
    g.off = g.wall ? se[comp] : 0;
    g.ih2 = 1.0 / (h * h);
    return g;
}

int64_t helm_unknowns(const HelmGeo& g) { return (int64_t)g.m[0] * g.m[1] * g.m[2]; }
int64_t helm_faces(const HelmGeo& g) { return (int64_t)g.e[0] * g.e[1] * g.e[2]; }

int64_t launch_helm_init(const HelmGeo& g, const double* un, const double* nu, double tau, double* us,
                         double* partials, cudaStream_t st, FinSpec fin) {
    const int64_t n = helm_unknowns(g);
    const int nb = elementwise_blocks(n);
    helm_init_kernel<<<nb, kRedThreads, 0, st>>>(g, n, un, nu, tau, us, partials, fin);
    count_launch();
    return nb;
}

int64_t launch_helm_residual(const HelmGeo& g, const double* un, const double* nu, double tau, const double* x,
                             double* r, double* z, double* partials, cudaStream_t st, FinSpec fin) {
    const int64_t n = helm_unknowns(g);
    const int nb = elementwise_blocks(n);
    helm_residual_kernel<<<nb, kRedThreads, 0, st>>>(g, n, un, nu, tau, x, r, z, partials, fin);
    count_launch();
    return nb;
}

int64_t launch_helm_matvec_dot(const HelmGeo& g, const double* nu, double tau, const double* d, double* q,
                               double* partials, cudaStream_t st, FinSpec fin) {
    const int64_t n = helm_unknowns(g);
    const int nb = elementwise_blocks(n);
    helm_matvec_dot_kernel<<<nb, kRedThreads, 0, st>>>(g, n, nu, tau, d, q, partials, fin);
    count_launch();
    return nb;
}

int64_t launch_helm_update(const HelmGeo& g, const double* nu, double tau, const Scal* s, const double* d,
                           const double* q, double* x, double* r, double* z, double* partials, cudaStream_t st,
                           FinSpec fin) {
    const int64_t n = helm_unknowns(g);
    const int nb = elementwise_blocks(n);
    helm_update_kernel<<<nb, kRedThreads, 0, st>>>(g, n, nu, tau, s, d, q, x, r, z, partials, fin);
    count_launch();
    return nb;
}

void launch_helm_face_nu(const HelmGeo& g, const Geo& g0, const double* C, double mu1, double mu2, double rho1,
                         double rho2, double* nu, cudaStream_t st) {
    const int64_t nfull = helm_faces(g);
    helm_face_nu_kernel<<<elementwise_blocks(nfull), kRedThreads, 0, st>>>(g, nfull, g0.nx, g0.ny, C, mu1, mu2,
                                                                           rho1, rho2, nu);
    count_launch();
}

}  // namespace paris
