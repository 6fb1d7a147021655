// Fused red-black Gauss-Seidel sweep (both colours in one pass over memory).
//
// The paper's red-black Gauss-Seidel with over-relaxation (Eq. eq:beta_pressure,
// Sec. 3.7.1) updates all cells of one colour, then all cells of the other.
// On the GPU the two colour passes each stream the coefficient and solution
// arrays from HBM; this kernel does the whole sweep in one pass:
//
//   * a CTA owns a TX x TY tile of an (x, y) plane and a slab of z-planes and
//     marches through the slab plane by plane;
//   * at step k it updates the FIRST colour on plane k over the tile plus a
//     one-cell halo (recomputed redundantly by the neighbouring CTAs, so no CTA
//     waits for another), then the SECOND colour on plane k-1 over the tile,
//     using the first-colour values just computed;
//   * old solution planes (tile + 2-cell halo) and new first-colour planes
//     (tile + 1-cell halo) live in 3-plane shared-memory rings;
//   * input and output are separate arrays (ping-pong), so halo reads never
//     see another CTA's updates.
//
// The result is bit-identical to one pass of each colour in place (same
// arithmetic in the same order).  With zero_init the incoming solution is
// taken as zero and never read.
#include "kernels.cuh"

namespace paris {

namespace {

constexpr int FTX = 30, FTY = 6;           // tile owned by one CTA
constexpr int HX1 = FTX + 2, HY1 = FTY + 2; // tile + 1 halo (= thread block)
constexpr int HX2 = FTX + 4, HY2 = FTY + 4; // tile + 2 halo
constexpr int FZ = 32;                      // z-planes per slab

__device__ inline int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// coefficient of the - and + face along each axis of cell (i,j,k) (walls: 0)
template <typename T>
__device__ inline void cell_coefs(const Geo& g, const Coef<T>& cf, int i, int j, int k, T b[6]) {
    AxisNb ax = axis_nb(i, g.nx, g.wx), ay = axis_nb(j, g.ny, g.wy), az = axis_nb(k, g.nz, g.wz);
    b[0] = ax.wm ? T(0) : cf.bx[g.fx(i, j, k)];
    b[1] = ax.wp ? T(0) : cf.bx[g.fx(ax.fp, j, k)];
    b[2] = ay.wm ? T(0) : cf.by[g.fy(i, j, k)];
    b[3] = ay.wp ? T(0) : cf.by[g.fy(i, ay.fp, k)];
    b[4] = az.wm ? T(0) : cf.bz[g.fz(i, j, k)];
    b[5] = az.wp ? T(0) : cf.bz[g.fz(i, j, az.fp)];
}

// map a (possibly out-of-range) coordinate to a cell index along one axis:
// periodic axes wrap; wall axes return -1 outside the domain.
__device__ inline int axis_cell(int i, int n, int wall) {
    if (i >= 0 && i < n) return i;
    return wall ? -1 : wrap(i, n);
}

}  // namespace

template <typename T>
__global__ void __launch_bounds__(HX1* HY1)
    rbgs_fused_kernel(Geo g, Coef<T> cf, const T* __restrict__ wdiag, const T* __restrict__ f,
                      const T* __restrict__ xin, T* __restrict__ xout, int first, T omega,
                      int zero_init, int use_w) {
    __shared__ T xo[3][HY2][HX2];  // old solution, planes k-1, k, k+1 (ring by plane % 3)
    __shared__ T xn[3][HY1][HX1];  // first-colour values, planes k-2, k-1, k

    const int tx = threadIdx.x, ty = threadIdx.y;  // position in the tile + 1 halo
    const int tid = ty * HX1 + tx;
    const int i0 = blockIdx.x * FTX, j0 = blockIdx.y * FTY;
    const int z0 = blockIdx.z * FZ, z1 = min(z0 + FZ, g.nz);
    const T hs = T(1) / cf.scale;

    // my cell in the tile + 1 halo region
    const int gi = axis_cell(i0 - 1 + tx, g.nx, g.wx);
    const int gj = axis_cell(j0 - 1 + ty, g.ny, g.wy);
    const bool interior = tx >= 1 && tx <= FTX && ty >= 1 && ty <= FTY && (i0 - 1 + tx) < g.nx &&
                          (j0 - 1 + ty) < g.ny;

    auto load_old = [&](int kk) {  // plane kk (unwrapped) of the old solution into the ring
        const int gk = axis_cell(kk, g.nz, g.wz);
        T* dst = &xo[((kk % 3) + 3) % 3][0][0];
        for (int e = tid; e < HY2 * HX2; e += HX1 * HY1) {
            const int ey = e / HX2, ex = e % HX2;
            const int ii = axis_cell(i0 - 2 + ex, g.nx, g.wx);
            const int jj = axis_cell(j0 - 2 + ey, g.ny, g.wy);
            T v = T(0);
            if (!zero_init && gk >= 0 && ii >= 0 && jj >= 0) v = xin[g.cidx(ii, jj, gk)];
            dst[e] = v;
        }
    };

    // colour of global (unwrapped) coordinates: parity of i+j+k; the grid
    // dimensions may be odd along a periodic axis, so use the wrapped indices
    auto colour_of = [&](int ii, int jj, int kk) { return (ii + jj + kk) & 1; };

    // GS update of cell (gi, gj, gk) from its six neighbours' values (same
    // arithmetic as the single-colour kernel); zi: the zero-start formula
    auto update = [&](bool zi, int gk, T xc, T xm, T xp, T ym, T yp, T zm, T zp) -> T {
        T b[6];
        cell_coefs(g, cf, gi, gj, gk, b);
        const int64_t c = g.cidx(gi, gj, gk);
        T acc = f[c] * hs;
        acc = fma(b[0], xm, acc);
        acc = fma(b[1], xp, acc);
        acc = fma(b[2], ym, acc);
        acc = fma(b[3], yp, acc);
        acc = fma(b[4], zm, acc);
        acc = fma(b[5], zp, acc);
        T w;
        if (use_w) {
            w = wdiag[c];
        } else {
            const T d = ((b[0] + b[1]) + (b[2] + b[3])) + (b[4] + b[5]);
            w = d > T(0) ? T(1) / d : T(0);
        }
        if (zi) return omega * w * acc;  // first colour from a zero solution
        return fma(omega, fma(w, acc, -xc), xc);
    };

    // prologue: old planes z0-2 .. z0 (the ring holds three planes)
    load_old(z0 - 2);
    load_old(z0 - 1);
    for (int k = z0 - 1; k <= z1; ++k) {
        // old plane k+1 replaces plane k-2
        load_old(k + 1);
        __syncthreads();
        // ---- first colour on plane k over the tile + 1 halo
        const int gk = axis_cell(k, g.nz, g.wz);
        const int sk = ((k % 3) + 3) % 3, skm = (((k - 1) % 3) + 3) % 3, skp = (((k + 1) % 3) + 3) % 3;
        {
            T v = T(0);
            if (gk >= 0 && gi >= 0 && gj >= 0 && colour_of(gi, gj, gk) == first) {
                const int sy = ty + 1, sx = tx + 1;  // position in the halo-2 arrays
                v = update(zero_init != 0, gk, xo[sk][sy][sx], xo[sk][sy][sx - 1], xo[sk][sy][sx + 1],
                           xo[sk][sy - 1][sx], xo[sk][sy + 1][sx], xo[skm][sy][sx], xo[skp][sy][sx]);
            } else if (gk >= 0 && gi >= 0 && gj >= 0) {
                v = xo[sk][ty + 1][tx + 1];  // second colour: old value (not used for updates)
            }
            xn[sk][ty][tx] = v;
        }
        __syncthreads();
        // ---- second colour on plane k-1 over the tile; write the tile's plane k-1
        const int kb = k - 1;
        if (kb >= z0 && kb < z1 && interior) {
            const int gkb = kb;  // inside the slab, always a real plane
            const int sb = (((kb) % 3) + 3) % 3, sbm = (((kb - 1) % 3) + 3) % 3, sbp = sk;
            T out;
            if (colour_of(gi, gj, gkb) != first) {
                const T xc = xo[sb][ty + 1][tx + 1];
                out = update(false, gkb, xc, xn[sb][ty][tx - 1], xn[sb][ty][tx + 1], xn[sb][ty - 1][tx],
                             xn[sb][ty + 1][tx], xn[sbm][ty][tx], xn[sbp][ty][tx]);
            } else {
                out = xn[sb][ty][tx];
            }
            xout[g.cidx(gi, gj, gkb)] = out;
        }
        // the next step's load replaces the old plane k-1 read just above:
        // wait for every reader first
        __syncthreads();
    }
}

template <typename T>
void launch_rbgs_fused(const Geo& g, const Coef<T>& cf, const T* w, const T* f, const T* xin,
                       T* xout, int first_color, double omega, bool zero_init, bool use_w,
                       cudaStream_t st) {
    dim3 gr((g.nx + FTX - 1) / FTX, (g.ny + FTY - 1) / FTY, (g.nz + FZ - 1) / FZ);
    rbgs_fused_kernel<T><<<gr, dim3(HX1, HY1), 0, st>>>(g, cf, w, f, xin, xout, first_color,
                                                         (T)omega, zero_init ? 1 : 0, use_w ? 1 : 0);
    count_launch();
}

template void launch_rbgs_fused<float>(const Geo&, const Coef<float>&, const float*, const float*,
                                       const float*, float*, int, double, bool, bool, cudaStream_t);
template void launch_rbgs_fused<double>(const Geo&, const Coef<double>&, const double*,
                                        const double*, const double*, double*, int, double, bool,
                                        bool, cudaStream_t);

}  // namespace paris
