// Adjoint (reverse-mode derivative) of the projection step.
//
// The paper has no adjoint; it follows from Eqs. fotm and poisson.  With
// B = diag(beta), D the divergence and G the face gradient (D = -G^T on
// non-wall faces), the projection is u = u* - B G L^{-1} D u* (dt cancels),
// L = D B G.  For a loss with gradient g = dLoss/du, and q the mean-free
// solution of L q = D (B g):
//   dLoss/du*_f   = g_f - (G q)_f
//   dLoss/dbeta_f = dt (G p)_f ((G q)_f - g_f)
//   dLoss/dC_c    = sum over the faces f of c of dLoss/dbeta_f dbeta_f/dC_c,
//                   dbeta_f/dC_c = -beta_f^2 (rho1 - rho2) / 2
// (beta_f = 2/(rho_L + rho_R), rho = rho1 C + rho2 (1 - C)).  Wall faces carry
// neither velocity nor coefficient, so every derivative there is zero.
#include "kernels.cuh"

namespace paris {

namespace {
constexpr int kTX = 32, kTY = 8, kZ = 8;
}

// c = D (B g) / 1: the divergence of the face field beta*g (walls carry no
// flux), with block partials (sum, max |c|, non-finite count).
__global__ void __launch_bounds__(kTX* kTY)
    weighted_div_kernel(Geo g, const double* __restrict__ bx, const double* __restrict__ by,
                        const double* __restrict__ bz, const double* __restrict__ gx,
                        const double* __restrict__ gy, const double* __restrict__ gz, double inv_h,
                        double* __restrict__ out, double* partials) {
    const int i = blockIdx.x * kTX + threadIdx.x;
    const int j = blockIdx.y * kTY + threadIdx.y;
    double acc[3] = {0.0, 0.0, 0.0};
    if (i < g.nx && j < g.ny) {
        const int k0 = blockIdx.z * kZ, k1 = min(k0 + kZ, g.nz);
        for (int k = k0; k < k1; ++k) {
            AxisNb ax = axis_nb(i, g.nx, g.wx), ay = axis_nb(j, g.ny, g.wy), az = axis_nb(k, g.nz, g.wz);
            const int64_t fxp = g.fx(ax.fp, j, k), fxm = g.fx(i, j, k);
            const int64_t fyp = g.fy(i, ay.fp, k), fym = g.fy(i, j, k);
            const int64_t fzp = g.fz(i, j, az.fp), fzm = g.fz(i, j, k);
            const double up = ax.wp ? 0.0 : bx[fxp] * gx[fxp];
            const double um = ax.wm ? 0.0 : bx[fxm] * gx[fxm];
            const double vp = ay.wp ? 0.0 : by[fyp] * gy[fyp];
            const double vm = ay.wm ? 0.0 : by[fym] * gy[fym];
            const double wp = az.wp ? 0.0 : bz[fzp] * gz[fzp];
            const double wm = az.wm ? 0.0 : bz[fzm] * gz[fzm];
            const double c = (((up - um) + (vp - vm)) + (wp - wm)) * inv_h;
            out[g.cidx(i, j, k)] = c;
            acc[0] += c;
            acc[1] = fmax(acc[1], fabs(c));
            acc[2] += isfinite(c) ? 0.0 : 1.0;
        }
    }
    const int op[3] = {0, 1, 0};
    const int64_t blk = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    block_reduce_store<3>(acc, op, partials, blk, threadIdx.y * kTX + threadIdx.x);
}

int64_t launch_weighted_div(const Geo& g, const double* bx, const double* by, const double* bz,
                            const double* gx, const double* gy, const double* gz, double inv_h,
                            double* out, double* partials, cudaStream_t st) {
    dim3 gr((g.nx + kTX - 1) / kTX, (g.ny + kTY - 1) / kTY, (g.nz + kZ - 1) / kZ);
    weighted_div_kernel<<<gr, dim3(kTX, kTY), 0, st>>>(g, bx, by, bz, gx, gy, gz, inv_h, out, partials);
    count_launch();
    return (int64_t)gr.x * gr.y * gr.z;
}

// Per face: gq = (q_R - q_L)/h, gp = (p_R - p_L)/h;
//   gus = g - gq,  gbeta = dt gp (gq - g);  both 0 on wall faces.
// One thread per cell handles its - faces (and the + wall face of the last
// cell along a wall axis).
__global__ void adjoint_faces_kernel(Geo g, const double* __restrict__ p, const double* __restrict__ q,
                                     double inv_h, double dt, const double* __restrict__ gx,
                                     const double* __restrict__ gy, const double* __restrict__ gz,
                                     double* __restrict__ usx, double* __restrict__ usy,
                                     double* __restrict__ usz, double* __restrict__ bbx,
                                     double* __restrict__ bby, double* __restrict__ bbz) {
    const int i = blockIdx.x * kTX + threadIdx.x;
    const int j = blockIdx.y * kTY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const int64_t c = g.cidx(i, j, k);
    const double pc = p[c], qc = q[c];
    AxisNb ax = axis_nb(i, g.nx, g.wx), ay = axis_nb(j, g.ny, g.wy), az = axis_nb(k, g.nz, g.wz);
    auto face = [&](bool wall, int64_t f, int64_t left, const double* gin, double* us, double* bb) {
        if (wall) {
            us[f] = 0.0;
            bb[f] = 0.0;
            return;
        }
        const double gq = (qc - q[left]) * inv_h;
        const double gp = (pc - p[left]) * inv_h;
        const double gv = gin[f];
        us[f] = gv - gq;
        bb[f] = dt * gp * (gq - gv);
    };
    face(ax.wm, g.fx(i, j, k), g.cidx(ax.m, j, k), gx, usx, bbx);
    face(ay.wm, g.fy(i, j, k), g.cidx(i, ay.m, k), gy, usy, bby);
    face(az.wm, g.fz(i, j, k), g.cidx(i, j, az.m), gz, usz, bbz);
    if (g.wx && i == g.nx - 1) { usx[g.fx(g.nx, j, k)] = 0.0; bbx[g.fx(g.nx, j, k)] = 0.0; }
    if (g.wy && j == g.ny - 1) { usy[g.fy(i, g.ny, k)] = 0.0; bby[g.fy(i, g.ny, k)] = 0.0; }
    if (g.wz && k == g.nz - 1) { usz[g.fz(i, j, g.nz)] = 0.0; bbz[g.fz(i, j, g.nz)] = 0.0; }
}

void launch_adjoint_faces(const Geo& g, const double* p, const double* q, double inv_h, double dt,
                          const double* gx, const double* gy, const double* gz, double* usx,
                          double* usy, double* usz, double* bbx, double* bby, double* bbz,
                          cudaStream_t st) {
    dim3 gr((g.nx + kTX - 1) / kTX, (g.ny + kTY - 1) / kTY, g.nz);
    adjoint_faces_kernel<<<gr, dim3(kTX, kTY), 0, st>>>(g, p, q, inv_h, dt, gx, gy, gz, usx, usy, usz,
                                                         bbx, bby, bbz);
    count_launch();
}

// dLoss/dC_c = -(rho1 - rho2)/2 * sum over the six non-wall faces of c of
// gbeta_f beta_f^2 (gather: one thread per cell, no atomics).
__global__ void face_coeffs_adjoint_kernel(Geo g, double half_drho, const double* __restrict__ bx,
                                           const double* __restrict__ by,
                                           const double* __restrict__ bz,
                                           const double* __restrict__ gbx,
                                           const double* __restrict__ gby,
                                           const double* __restrict__ gbz, double* __restrict__ gC) {
    const int i = blockIdx.x * kTX + threadIdx.x;
    const int j = blockIdx.y * kTY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    AxisNb ax = axis_nb(i, g.nx, g.wx), ay = axis_nb(j, g.ny, g.wy), az = axis_nb(k, g.nz, g.wz);
    auto term = [](bool wall, const double* b, const double* gb, int64_t f) {
        if (wall) return 0.0;
        const double bf = b[f];
        return gb[f] * bf * bf;
    };
    double s = term(ax.wm, bx, gbx, g.fx(i, j, k)) + term(ax.wp, bx, gbx, g.fx(ax.fp, j, k));
    s += term(ay.wm, by, gby, g.fy(i, j, k)) + term(ay.wp, by, gby, g.fy(i, ay.fp, k));
    s += term(az.wm, bz, gbz, g.fz(i, j, k)) + term(az.wp, bz, gbz, g.fz(i, j, az.fp));
    gC[g.cidx(i, j, k)] = -half_drho * s;
}

void launch_face_coeffs_adjoint(const Geo& g, double rho1, double rho2, const double* bx,
                                const double* by, const double* bz, const double* gbx,
                                const double* gby, const double* gbz, double* gC, cudaStream_t st) {
    dim3 gr((g.nx + kTX - 1) / kTX, (g.ny + kTY - 1) / kTY, g.nz);
    face_coeffs_adjoint_kernel<<<gr, dim3(kTX, kTY), 0, st>>>(g, 0.5 * (rho1 - rho2), bx, by, bz, gbx,
                                                               gby, gbz, gC);
    count_launch();
}

}  // namespace paris
