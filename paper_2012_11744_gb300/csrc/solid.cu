// Solid cells ("Lego" solids, Sec. 3.8).
//
// A cell flag s (1 outside the solid, 0 inside, one byte per cell, the
// caller's device array) defines link flags on the faces: a face is open
// when both of its cells are fluid, s_f = s_L s_R (the paper blocks the
// velocity and the pressure correction on the solid region and on its
// boundary).  The library applies them in three places:
//   * the face coefficients: beta_f = 0 on closed faces (the pressure
//     coefficients A1..A6 zeroed, A7 their sum), so p sees a Neumann
//     condition on the solid's boundary;
//   * the divergence: closed faces carry no flux, whatever u* holds there;
//   * the velocity correction: u = 0 on closed faces (the blocking done
//     each time the velocity is updated).
// Solid cells then have no open face.  Their pressure is not determined by
// the system; the solve keeps it out of the gauge and reports 0 there, the
// fluid cells' pressure having zero mean.
#include "kernels.cuh"

namespace paris {

namespace {

constexpr int kTX = 32, kTY = 8;

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Thread per cell (i, j, k): the - face of each axis (face i between cells
// i-1, wrapped, and i); a closed face gets beta = 0 and u = 0 (pointers may
// be null).  Wall faces are left alone: they are closed already.
__global__ void __launch_bounds__(kTX* kTY) link_block_kernel(Geo g, const unsigned char* __restrict__ s,
                                                             double* bx, double* by, double* bz, double* u,
                                                             double* v, double* w) {
    const int i = blockIdx.x * kTX + threadIdx.x, j = blockIdx.y * kTY + threadIdx.y, k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const bool sc = s[g.cidx(i, j, k)] != 0;
    if (!(g.wx && i == 0)) {
        if (!sc || !s[g.cidx(wrap(i - 1, g.nx), j, k)]) {
            const int64_t f = g.fx(i, j, k);
            if (bx) bx[f] = 0.0;
            if (u) u[f] = 0.0;
        }
    }
    if (!(g.wy && j == 0)) {
        if (!sc || !s[g.cidx(i, wrap(j - 1, g.ny), k)]) {
            const int64_t f = g.fy(i, j, k);
            if (by) by[f] = 0.0;
            if (v) v[f] = 0.0;
        }
    }
    if (!(g.wz && k == 0)) {
        if (!sc || !s[g.cidx(i, j, wrap(k - 1, g.nz))]) {
            const int64_t f = g.fz(i, j, k);
            if (bz) bz[f] = 0.0;
            if (w) w[f] = 0.0;
        }
    }
}

// Eqs. cont2, incompdisc3 with closed faces carrying no flux: rhs = div/(h dt),
// 0 in solid cells; block partials (sum, max |rhs|, non-finite count).  A
// thread walks kZ planes of its column, so the grid is the divergence
// kernel's and fits the context's partial-sum slots.
constexpr int kZ = 8;

__global__ void __launch_bounds__(kTX* kTY) masked_divergence_kernel(Geo g, const unsigned char* __restrict__ s,
                                                                    const double* __restrict__ u,
                                                                    const double* __restrict__ v,
                                                                    const double* __restrict__ w, double inv_hdt,
                                                                    double* __restrict__ rhs, double* partials,
                                                                    FinSpec fin) {
    const int i = blockIdx.x * kTX + threadIdx.x, j = blockIdx.y * kTY + threadIdx.y;
    const int tid = threadIdx.y * kTX + threadIdx.x;
    double sum = 0.0;
    unsigned long long bmax = 0;
    unsigned nf = 0;
    if (i < g.nx && j < g.ny) {
        const int k0 = blockIdx.z * kZ, k1 = min(k0 + kZ, g.nz);
        for (int k = k0; k < k1; ++k) {
            const int64_t c = g.cidx(i, j, k);
            double b = 0.0;
            if (s[c]) {
                auto open = [&](int ii, int jj, int kk) { return s[g.cidx(ii, jj, kk)] != 0; };
                const bool xm = !(g.wx && i == 0) && open(wrap(i - 1, g.nx), j, k);
                const bool xp = !(g.wx && i == g.nx - 1) && open(wrap(i + 1, g.nx), j, k);
                const bool ym = !(g.wy && j == 0) && open(i, wrap(j - 1, g.ny), k);
                const bool yp = !(g.wy && j == g.ny - 1) && open(i, wrap(j + 1, g.ny), k);
                const bool zm = !(g.wz && k == 0) && open(i, j, wrap(k - 1, g.nz));
                const bool zp = !(g.wz && k == g.nz - 1) && open(i, j, wrap(k + 1, g.nz));
                const int ip = (i + 1 < g.nx || g.wx) ? i + 1 : 0, jp = (j + 1 < g.ny || g.wy) ? j + 1 : 0;
                const int kp = (k + 1 < g.nz || g.wz) ? k + 1 : 0;
                const double up = xp ? u[g.fx(ip, j, k)] : 0.0, um = xm ? u[g.fx(i, j, k)] : 0.0;
                const double vp = yp ? v[g.fy(i, jp, k)] : 0.0, vm = ym ? v[g.fy(i, j, k)] : 0.0;
                const double wp = zp ? w[g.fz(i, j, kp)] : 0.0, wm = zm ? w[g.fz(i, j, k)] : 0.0;
                b = (((up - um) + (vp - vm)) + (wp - wm)) * inv_hdt;
            }
            rhs[c] = b;
            sum += b;
            const unsigned long long kb = abs_key(b);
            bmax = kb > bmax ? kb : bmax;
            nf += key_nonfinite(kb);
        }
    }
    const int64_t blk = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    block_reduce_skc<double>(sum, bmax, nf, partials, blk, tid);
    finalize_last_block(partials, (int64_t)gridDim.x * gridDim.y * gridDim.z, fin, tid);
}

// Block partials of (sum over fluid cells of x, number of fluid cells).
__global__ void fluid_sum_kernel(int64_t n, const unsigned char* __restrict__ s, const double* __restrict__ x,
                                 double* partials) {
    double acc[2] = {0.0, 0.0};
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        if (s[c]) {
            acc[0] += x ? x[c] : 0.0;
            acc[1] += 1.0;
        }
    const int op[2] = {0, 0};
    block_reduce_store<2>(acc, op, partials, blockIdx.x, threadIdx.x);
}

// x <- x - (red[0] / red[1]) on fluid cells, 0 on solid cells
__global__ void fluid_gauge_kernel(int64_t n, const unsigned char* __restrict__ s, double* __restrict__ x,
                                   const Scal* sc) {
    const double m = sc->red[1] > 0.0 ? sc->red[0] / sc->red[1] : 0.0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        x[c] = s[c] ? x[c] - m : 0.0;
}

// x <- x - mean_b on fluid cells, 0 on solid cells (the divergence's mean,
// taken over the fluid cells)
__global__ void fluid_sub_mean_kernel(int64_t n, const unsigned char* __restrict__ s, double* __restrict__ x,
                                      const Scal* sc) {
    const double m = sc->mean_b;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        x[c] = s[c] ? x[c] - m : 0.0;
}

// x <- 0 on solid cells
__global__ void solid_zero_kernel(int64_t n, const unsigned char* __restrict__ s, double* __restrict__ x) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        if (!s[c]) x[c] = 0.0;
}

}  // namespace

void launch_link_block(const Geo& g, const unsigned char* s, double* bx, double* by, double* bz, double* u,
                       double* v, double* w, cudaStream_t st) {
    dim3 gr((g.nx + kTX - 1) / kTX, (g.ny + kTY - 1) / kTY, g.nz);
    link_block_kernel<<<gr, dim3(kTX, kTY), 0, st>>>(g, s, bx, by, bz, u, v, w);
    count_launch();
}

int64_t launch_masked_divergence(const Geo& g, const unsigned char* s, const double* u, const double* v,
                                 const double* w, double inv_hdt, double* rhs, double* partials, cudaStream_t st,
                                 FinSpec fin) {
    dim3 gr((g.nx + kTX - 1) / kTX, (g.ny + kTY - 1) / kTY, (g.nz + kZ - 1) / kZ);
    masked_divergence_kernel<<<gr, dim3(kTX, kTY), 0, st>>>(g, s, u, v, w, inv_hdt, rhs, partials, fin);
    count_launch();
    return (int64_t)gr.x * gr.y * gr.z;
}

void launch_fluid_gauge(int64_t n, const unsigned char* s, double* x, double* partials, Scal* sc, cudaStream_t st) {
    const int nb = elementwise_blocks(n);
    fluid_sum_kernel<<<nb, kRedThreads, 0, st>>>(n, s, x, partials);
    finalize(partials, nb, 2, 0, sc, FIN_STORE, 0.0, st);
    fluid_gauge_kernel<<<nb, kRedThreads, 0, st>>>(n, s, x, sc);
    count_launch(2);
}

void launch_solid_zero(int64_t n, const unsigned char* s, double* x, cudaStream_t st) {
    solid_zero_kernel<<<elementwise_blocks(n), kRedThreads, 0, st>>>(n, s, x);
    count_launch();
}

int64_t launch_fluid_count(int64_t n, const unsigned char* s, double* partials, Scal* sc, cudaStream_t st) {
    const int nb = elementwise_blocks(n);
    fluid_sum_kernel<<<nb, kRedThreads, 0, st>>>(n, s, nullptr, partials);
    finalize(partials, nb, 2, 0, sc, FIN_STORE, 0.0, st);
    count_launch();
    return nb;
}

}  // namespace paris

namespace paris {

void launch_fluid_sub_mean(int64_t n, const unsigned char* s, double* x, const Scal* sc, cudaStream_t st) {
    fluid_sub_mean_kernel<<<elementwise_blocks(n), kRedThreads, 0, st>>>(n, s, x, sc);
    count_launch();
}

// mean of x over the fluid cells into sc->mean_b (FIN_MEAN_FLUID)
void launch_fluid_mean(int64_t n, const unsigned char* s, const double* x, double* partials, Scal* sc,
                       cudaStream_t st) {
    const int nb = elementwise_blocks(n);
    fluid_sum_kernel<<<nb, kRedThreads, 0, st>>>(n, s, x, partials);
    finalize(partials, nb, 2, 0, sc, FIN_MEAN_FLUID, 0.0, st);
    count_launch();
}

}  // namespace paris

// ------------------------------------------------------ marker function ---
// Sec. 3.4.2, Eq. FrontMarker3: Lap_h I = D G_f is the projection's operator
// with beta = 1 on every face (0 on the wall faces).

namespace paris {

namespace {

__global__ void unit_beta_kernel(Geo g, int axis, int64_t n, double* __restrict__ b) {
    const int e0 = g.nx + (axis == 0 ? g.wx : 0), e1 = g.ny + (axis == 1 ? g.wy : 0);
    const int wall = axis == 0 ? g.wx : (axis == 1 ? g.wy : g.wz);
    const int na = axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz);
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n; f += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = f / e0;
        const int i = (int)(f - t * e0), j = (int)(t % e1), k = (int)(t / e1);
        const int p = axis == 0 ? i : (axis == 1 ? j : k);
        b[f] = (wall && (p == 0 || p == na)) ? 0.0 : 1.0;
    }
}

__global__ void add_constant_kernel(int64_t n, double* __restrict__ x, double a) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        x[c] += a;
}

}  // namespace

void launch_unit_beta(const Geo& g, double* bx, double* by, double* bz, cudaStream_t st) {
    double* b[3] = {bx, by, bz};
    for (int a = 0; a < 3; ++a) {
        const int64_t n = g.nface(a);
        unit_beta_kernel<<<elementwise_blocks(n), kRedThreads, 0, st>>>(g, a, n, b[a]);
    }
    count_launch(3);
}

void launch_add_constant(int64_t n, double* x, double a, cudaStream_t st) {
    add_constant_kernel<<<elementwise_blocks(n), kRedThreads, 0, st>>>(n, x, a);
    count_launch();
}

}  // namespace paris
