// Free-surface projections (Sec. 3.7.5 "Free-surface flow solver" and
// "Ensuring volume conservation").
//
// Both are projections on a subset of the cells with three classes per cell:
//   1  unknown   (the pressure is solved there),
//   2  Dirichlet (the pressure is given: the gas),
//   0  excluded  (a zero-gradient face towards it: Neumann).
// The face coefficient is beta between two unknown cells and 0 otherwise; a
// face from an unknown cell c to a Dirichlet cell at the distance theta h
// from c's node (Eq. mod_branches) adds beta/theta to c's diagonal (the
// operator's diagonal excess, Coef::sig) and beta/(theta h^2) p_s to its
// right-hand side, p_s the pressure on the interface.  The solve is the FP64
// multigrid-preconditioned CG with that excess on every level (no null space
// when every unknown region touches a Dirichlet cell).
//
// * Ghost-fluid solve in the liquid (Sec. 3.7.5): unknown = the cells with
//   C < 1/2 (C the gas fraction, 0 in the liquid), Dirichlet = the gas,
//   beta = 1/rho_l, p_s = p_gas + sigma (kappa_c + kappa_g)/2 (Eq.
//   Laplace_num, p_gas the gas cell's pressure from the polytropic law of
//   Eq. polygas).  The velocity correction (Eq. fotm) uses the same cut-face
//   gradients; faces between two gas cells are left as they are.
// * Phantom projection in two gas layers: unknown = the first two layers of
//   gas cells (through faces), excluded = the liquid (its faces keep their
//   solved velocities, zero gradient), Dirichlet = the gas beyond with
//   P = 0 at the cell centres (theta = 1); beta = 1, no dt; only the faces
//   between two non-liquid cells, one of them in the layers, are corrected.
#include "kernels.cuh"

namespace paris {

namespace {

constexpr int kTX = 32, kTY = 8;

__global__ void fs_liquid_classes_kernel(int64_t n, const double* __restrict__ C, unsigned char* __restrict__ cls) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        cls[c] = C[c] < 0.5 ? 1 : 2;
}

// The face neighbours of (i, j, k) in the order x-, x+, y-, y+, z-, z+;
// false where the face is a domain wall.
struct Nb6 {
    int64_t c[6];
    int64_t f[6];  // index of the shared face in its axis' face array
    bool ok[6];
};

__device__ __forceinline__ Nb6 nb6(const Geo& g, int i, int j, int k) {
    Nb6 q;
    const AxisNb ax = axis_nb(i, g.nx, g.wx), ay = axis_nb(j, g.ny, g.wy), az = axis_nb(k, g.nz, g.wz);
    q.c[0] = g.cidx(ax.m, j, k), q.f[0] = g.fx(i, j, k), q.ok[0] = !ax.wm;
    q.c[1] = g.cidx(ax.p, j, k), q.f[1] = g.fx(ax.fp, j, k), q.ok[1] = !ax.wp;
    q.c[2] = g.cidx(i, ay.m, k), q.f[2] = g.fy(i, j, k), q.ok[2] = !ay.wm;
    q.c[3] = g.cidx(i, ay.p, k), q.f[3] = g.fy(i, ay.fp, k), q.ok[3] = !ay.wp;
    q.c[4] = g.cidx(i, j, az.m), q.f[4] = g.fz(i, j, k), q.ok[4] = !az.wm;
    q.c[5] = g.cidx(i, j, az.p), q.f[5] = g.fz(i, j, az.fp), q.ok[5] = !az.wp;
    return q;
}

// Layer 1 of the gas (a liquid face neighbour): 0 liquid, 1 layer 1, 2 other gas.
__global__ void __launch_bounds__(kTX* kTY) fs_layer1_kernel(Geo g, const double* __restrict__ C,
                                                            unsigned char* __restrict__ tmp) {
    const int i = blockIdx.x * kTX + threadIdx.x, j = blockIdx.y * kTY + threadIdx.y, k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const int64_t c = g.cidx(i, j, k);
    unsigned char v = 0;
    if (!(C[c] < 0.5)) {
        const Nb6 q = nb6(g, i, j, k);
        bool touch = false;
        for (int s = 0; s < 6; ++s) touch = touch || (q.ok[s] && C[q.c[s]] < 0.5);
        v = touch ? 1 : 2;
    }
    tmp[c] = v;
}

// Layer 2 (a face neighbour in layer 1) joins layer 1 as the unknowns:
// 0 liquid (excluded), 1 the two layers, 2 the gas beyond (Dirichlet).
__global__ void __launch_bounds__(kTX* kTY) fs_layer2_kernel(Geo g, const unsigned char* __restrict__ tmp,
                                                            unsigned char* __restrict__ cls) {
    const int i = blockIdx.x * kTX + threadIdx.x, j = blockIdx.y * kTY + threadIdx.y, k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const int64_t c = g.cidx(i, j, k);
    unsigned char v = tmp[c];
    if (v == 2) {
        const Nb6 q = nb6(g, i, j, k);
        bool touch = false;
        for (int s = 0; s < 6; ++s) touch = touch || (q.ok[s] && tmp[q.c[s]] == 1);
        if (touch) v = 1;
    }
    cls[c] = v;
}

__device__ __forceinline__ double face_theta(const double* const th[3], int s, int64_t f) {
    const double* t = th[s >> 1];
    return t ? t[f] : 1.0;
}

// p_s on the face between the unknown cell c and the Dirichlet cell d (Eq. Laplace_num)
__device__ __forceinline__ double surface_p(const double* __restrict__ pd, const double* __restrict__ kappa,
                                            double sigma, int64_t c, int64_t d) {
    const double pg = pd ? pd[d] : 0.0;
    return kappa ? pg + sigma * (0.5 * (kappa[c] + kappa[d])) : pg;
}

// Thread per cell: beta on its - faces (and the + wall faces), its diagonal
// excess sig_c = sum over Dirichlet faces of beta/theta and the Dirichlet
// part of its right-hand side gd_c = 1/h^2 sum of beta/theta p_s.
__global__ void __launch_bounds__(kTX* kTY) fs_setup_kernel(Geo g, const unsigned char* __restrict__ cls,
                                                           double beta, const double* thx, const double* thy,
                                                           const double* thz, const double* __restrict__ pd,
                                                           const double* __restrict__ kappa, double sigma,
                                                           double ih2, double* __restrict__ bx,
                                                           double* __restrict__ by, double* __restrict__ bz,
                                                           double* __restrict__ sig, double* __restrict__ gd) {
    const int i = blockIdx.x * kTX + threadIdx.x, j = blockIdx.y * kTY + threadIdx.y, k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const int64_t c = g.cidx(i, j, k);
    const Nb6 q = nb6(g, i, j, k);
    const unsigned char cc = cls[c];
    double* const b[3] = {bx, by, bz};
    const double* const th[3] = {thx, thy, thz};
    for (int a = 0; a < 3; ++a) {
        const int s = 2 * a;  // the - face
        b[a][q.f[s]] = (q.ok[s] && cc == 1 && cls[q.c[s]] == 1) ? beta : 0.0;
        if (!q.ok[s + 1]) b[a][q.f[s + 1]] = 0.0;  // the + wall face
    }
    double sg = 0.0, rd = 0.0;
    if (cc == 1) {
        for (int s = 0; s < 6; ++s) {
            if (!q.ok[s] || cls[q.c[s]] != 2) continue;
            const double cf = beta / face_theta(th, s, q.f[s]);
            sg += cf;
            rd = fma(cf, surface_p(pd, kappa, sigma, c, q.c[s]), rd);
        }
    }
    sig[c] = sg;
    gd[c] = rd * ih2;
}

// rhs = div u / (h dt) - gd on the unknown cells (wall faces carry no flux),
// 0 elsewhere; gd is read from rhs and overwritten.
__global__ void __launch_bounds__(kTX* kTY) fs_rhs_kernel(Geo g, const unsigned char* __restrict__ cls,
                                                         const double* __restrict__ u, const double* __restrict__ v,
                                                         const double* __restrict__ w, double inv_hdt,
                                                         double* __restrict__ rhs) {
    const int i = blockIdx.x * kTX + threadIdx.x, j = blockIdx.y * kTY + threadIdx.y, k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const int64_t c = g.cidx(i, j, k);
    if (cls[c] != 1) {
        rhs[c] = 0.0;
        return;
    }
    const Nb6 q = nb6(g, i, j, k);
    const double* const uu[3] = {u, v, w};
    double d = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (q.ok[2 * a + 1]) d += uu[a][q.f[2 * a + 1]];
        if (q.ok[2 * a]) d -= uu[a][q.f[2 * a]];
    }
    rhs[c] = fma(d, inv_hdt, -rhs[c]);
}

// Eq. fotm on the faces touching an unknown cell with the cut-face gradients
// of Eq. mod_branches: u -= coef (p_hi - p_lo)/theta with p_s in place of a
// Dirichlet cell's value; faces touching an excluded cell, faces between
// two Dirichlet cells and (zero_walls = 0) wall faces are left alone.
__global__ void __launch_bounds__(kTX* kTY) fs_project_kernel(Geo g, const unsigned char* __restrict__ cls,
                                                             const double* thx, const double* thy,
                                                             const double* thz, const double* __restrict__ p,
                                                             const double* __restrict__ pd,
                                                             const double* __restrict__ kappa, double sigma,
                                                             double coef, int zero_walls, double* u, double* v,
                                                             double* w) {
    const int i = blockIdx.x * kTX + threadIdx.x, j = blockIdx.y * kTY + threadIdx.y, k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const int64_t c = g.cidx(i, j, k);
    const Nb6 q = nb6(g, i, j, k);
    double* const uu[3] = {u, v, w};
    const double* const th[3] = {thx, thy, thz};
    const unsigned char ch = cls[c];
    for (int a = 0; a < 3; ++a) {
        const int s = 2 * a;
        if (!q.ok[s + 1] && zero_walls) uu[a][q.f[s + 1]] = 0.0;
        if (!q.ok[s]) {
            if (zero_walls) uu[a][q.f[s]] = 0.0;
            continue;
        }
        // the - face: lower cell q.c[s], upper cell c
        const int64_t lo = q.c[s];
        const unsigned char cl = cls[lo];
        if (cl == 0 || ch == 0 || (cl != 1 && ch != 1)) continue;
        double dp;
        if (cl == 1 && ch == 1)
            dp = p[c] - p[lo];
        else if (cl == 1)
            dp = (surface_p(pd, kappa, sigma, lo, c) - p[lo]) / face_theta(th, s, q.f[s]);
        else
            dp = (p[c] - surface_p(pd, kappa, sigma, c, lo)) / face_theta(th, s, q.f[s]);
        uu[a][q.f[s]] = fma(-coef, dp, uu[a][q.f[s]]);
    }
}

// p outside the unknowns: the Dirichlet value (or 0)
__global__ void fs_fill_kernel(int64_t n, const unsigned char* __restrict__ cls, const double* __restrict__ pd,
                               double* __restrict__ p) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const unsigned char v = cls[c];
        if (v != 1) p[c] = (v == 2 && pd) ? pd[c] : 0.0;
    }
}

dim3 cell_grid(const Geo& g) { return dim3((g.nx + kTX - 1) / kTX, (g.ny + kTY - 1) / kTY, g.nz); }

}  // namespace

void launch_fs_liquid_classes(const Geo& g, const double* C, unsigned char* cls, cudaStream_t st) {
    fs_liquid_classes_kernel<<<elementwise_blocks(g.ncell()), kRedThreads, 0, st>>>(g.ncell(), C, cls);
    count_launch();
}

void launch_fs_gas_layers(const Geo& g, const double* C, unsigned char* tmp, unsigned char* cls, cudaStream_t st) {
    fs_layer1_kernel<<<cell_grid(g), dim3(kTX, kTY), 0, st>>>(g, C, tmp);
    fs_layer2_kernel<<<cell_grid(g), dim3(kTX, kTY), 0, st>>>(g, tmp, cls);
    count_launch(2);
}

void launch_fs_setup(const Geo& g, const unsigned char* cls, double beta, const double* const theta[3],
                     const double* pd, const double* kappa, double sigma, double h, double* bx, double* by,
                     double* bz, double* sig, double* gd, cudaStream_t st) {
    fs_setup_kernel<<<cell_grid(g), dim3(kTX, kTY), 0, st>>>(g, cls, beta, theta[0], theta[1], theta[2], pd, kappa,
                                                             sigma, 1.0 / (h * h), bx, by, bz, sig, gd);
    count_launch();
}

void launch_fs_rhs(const Geo& g, const unsigned char* cls, const double* u, const double* v, const double* w,
                   double inv_hdt, double* rhs, cudaStream_t st) {
    fs_rhs_kernel<<<cell_grid(g), dim3(kTX, kTY), 0, st>>>(g, cls, u, v, w, inv_hdt, rhs);
    count_launch();
}

void launch_fs_project(const Geo& g, const unsigned char* cls, const double* const theta[3], const double* p,
                       const double* pd, const double* kappa, double sigma, double coef, bool zero_walls,
                       double* u, double* v, double* w, cudaStream_t st) {
    fs_project_kernel<<<cell_grid(g), dim3(kTX, kTY), 0, st>>>(g, cls, theta[0], theta[1], theta[2], p, pd, kappa,
                                                               sigma, coef, zero_walls ? 1 : 0, u, v, w);
    count_launch();
}

void launch_fs_fill(const Geo& g, const unsigned char* cls, const double* pd, double* p, cudaStream_t st) {
    fs_fill_kernel<<<elementwise_blocks(g.ncell()), kRedThreads, 0, st>>>(g.ncell(), cls, pd, p);
    count_launch();
}

}  // namespace paris
