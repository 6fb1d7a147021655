// Fused red-black Gauss-Seidel sweep (both colours in one pass over memory).
//
// The paper's red-black Gauss-Seidel with over-relaxation (Eq. eq:beta_pressure,
// Sec. 3.7.1) updates all cells of one colour, then all cells of the other.
// On the GPU the two colour passes each stream the coefficient and solution
// arrays from HBM; this kernel does the whole sweep in one pass:
//
//   * a CTA owns a FTX x FTY tile of an (x, y) plane and a slab of FZ
//     z-planes and marches through the slab plane by plane;
//   * at step k it updates the FIRST colour on plane k over the tile plus a
//     one-cell halo (recomputed redundantly by the neighbouring CTAs, so no CTA
//     waits for another), then the SECOND colour on plane k-1 over the tile,
//     using the first-colour values just computed;
//   * old solution planes (tile + 2-cell halo) and new first-colour planes
//     (tile + 1-cell halo) live in 3-plane shared-memory rings; each thread
//     prefetches its own cell's coefficients and right-hand side one plane
//     ahead in registers;
//   * input and output are separate arrays (ping-pong), so halo reads never
//     see another CTA's updates.
//
// The result is bit-identical to one in-place pass of each colour (same
// arithmetic in the same order) when every periodic axis has even length.
// With ZERO the incoming solution is taken as zero and never read.
// Indices are 32-bit: the host uses this kernel only for levels whose face
// arrays hold fewer than 2^31 entries (rbgs_fused_fits).
#include "kernels.cuh"

namespace paris {

namespace {

constexpr int FTX = 30, FTY = 14;              // tile owned by one CTA
constexpr int HX1 = FTX + 2, HY1 = FTY + 2;    // tile + 1 halo (= thread block)
constexpr int HX2 = FTX + 4, HY2 = FTY + 4;    // tile + 2 halo
constexpr int FZ = 32;                         // z-planes per slab
constexpr int NT = HX1 * HY1;                  // threads per CTA
constexpr int NE = (HY2 * HX2 + NT - 1) / NT;  // halo-2 elements per thread and plane

// periodic axes wrap; wall axes return -1 outside the domain
__device__ inline int axis_cell(int i, int n, int wall) {
    if (i >= 0 && i < n) return i;
    if (wall) return -1;
    i %= n;
    return i < 0 ? i + n : i;
}

// My cell's data on one plane: f/scale, the six face coefficients
// (x-, x+, y-, y+, z-, z+) and the inverse diagonal.
template <typename T>
struct CellData {
    T f, b[6], w;
};

}  // namespace

template <typename T, bool ZERO, bool USEW>
__global__ void __launch_bounds__(NT)
    rbgs_fused_kernel(Geo g, Coef<T> cf, const T* __restrict__ wdiag, const T* __restrict__ f,
                      const T* __restrict__ xin, T* __restrict__ xout, int first, T omega) {
    __shared__ T xo[3][HY2][HX2];  // old solution, planes k-1, k, k+1 (slots sm, s0, sp)
    __shared__ T xn[3][HY1][HX1];  // first-colour values, planes k-2, k-1, k (slots sp, sm, s0)

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * HX1 + tx;
    const int i0 = blockIdx.x * FTX, j0 = blockIdx.y * FTY;
    const int z0 = blockIdx.z * FZ, z1 = min(z0 + FZ, g.nz);
    const T hs = T(1) / cf.scale;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int plane = nx * ny;

    // ---- per-thread column set-up (once)
    const int gi = axis_cell(i0 - 1 + tx, nx, g.wx);
    const int gj = axis_cell(j0 - 1 + ty, ny, g.wy);
    const bool col_ok = gi >= 0 && gj >= 0;
    const bool interior = tx >= 1 && tx <= FTX && ty >= 1 && ty <= FTY && (i0 - 1 + tx) < nx &&
                          (j0 - 1 + ty) < ny;
    const int par = (gi + gj) & 1;
    const int col = gj * nx + gi;
    const int nxf = nx + g.wx, pxf = ny * nxf;  // x-face row length and plane stride
    const int pyf = (ny + g.wy) * nx;           // y-face plane stride
    const bool wxm = g.wx && gi == 0, wxp = g.wx && gi == nx - 1;
    const bool wym = g.wy && gj == 0, wyp = g.wy && gj == ny - 1;
    const int cxm = gj * nxf + gi;
    const int cxp = gj * nxf + ((gi + 1 < nx || g.wx) ? gi + 1 : 0);
    const int cym = gj * nx + gi;
    const int cyp = ((gj + 1 < ny || g.wy) ? gj + 1 : 0) * nx + gi;
    int eoff[NE];  // in-plane offsets of my halo-2 elements, -1 outside the domain
#pragma unroll
    for (int q = 0; q < NE; ++q) {
        const int e = tid + q * NT;
        eoff[q] = -1;
        if (e < HY2 * HX2) {
            const int ii = axis_cell(i0 - 2 + e % HX2, nx, g.wx);
            const int jj = axis_cell(j0 - 2 + e / HX2, ny, g.wy);
            if (ii >= 0 && jj >= 0) eoff[q] = jj * nx + ii;
        }
    }

    auto fetch_old = [&](int kk, T (&v)[NE]) {
        const int gk = axis_cell(kk, nz, g.wz);
#pragma unroll
        for (int q = 0; q < NE; ++q)
            v[q] = (!ZERO && gk >= 0 && eoff[q] >= 0) ? xin[gk * plane + eoff[q]] : T(0);
    };
    auto store_old = [&](int slot, const T (&v)[NE]) {
        T* dst = &xo[slot][0][0];
#pragma unroll
        for (int q = 0; q < NE; ++q) {
            const int e = tid + q * NT;
            if (e < HY2 * HX2) dst[e] = v[q];
        }
    };
    auto fetch_cell = [&](int kk, CellData<T>& d) {
        const int gk = axis_cell(kk, nz, g.wz);
        if (gk < 0 || !col_ok) return;
        const int kp = (gk + 1 < nz || g.wz) ? gk + 1 : 0;
        d.b[0] = wxm ? T(0) : cf.bx[gk * pxf + cxm];
        d.b[1] = wxp ? T(0) : cf.bx[gk * pxf + cxp];
        d.b[2] = wym ? T(0) : cf.by[gk * pyf + cym];
        d.b[3] = wyp ? T(0) : cf.by[gk * pyf + cyp];
        d.b[4] = (g.wz && gk == 0) ? T(0) : cf.bz[gk * plane + col];
        d.b[5] = (g.wz && gk == nz - 1) ? T(0) : cf.bz[kp * plane + col];
        const int c = gk * plane + col;
        d.f = f[c] * hs;
        if (USEW) {
            d.w = wdiag[c];
        } else {
            const T s6 = ((d.b[0] + d.b[1]) + (d.b[2] + d.b[3])) + (d.b[4] + d.b[5]);
            d.w = s6 > T(0) ? T(1) / s6 : T(0);
        }
    };
    // GS update from the six neighbours' values (same arithmetic, same order
    // as the single-colour kernel); zi: the zero-start formula
    auto update = [&](bool zi, const CellData<T>& d, T xc, T xm, T xp, T ym, T yp, T zm, T zp) -> T {
        T acc = d.f;
        acc = fma(d.b[0], xm, acc);
        acc = fma(d.b[1], xp, acc);
        acc = fma(d.b[2], ym, acc);
        acc = fma(d.b[3], yp, acc);
        acc = fma(d.b[4], zm, acc);
        acc = fma(d.b[5], zp, acc);
        if (zi) return omega * d.w * acc;
        return fma(omega, fma(d.w, acc, -xc), xc);
    };

    // At step k the xo ring holds old planes k-1, k, k+1 in slots sm, s0, sp
    // (plane k+1 is stored at the start of the step) and the xn ring holds the
    // first-colour planes k-2, k-1, k in slots sp, sm, s0.
    int sm = 0, s0 = 1, sp = 2;
    CellData<T> dm{}, dc{}, dn{};  // my cell on planes k-1, k, k+1
    T on[NE], onn[NE];             // old halo-2 planes k+1 and k+2
    {
        T tmp[NE];
        fetch_old(z0 - 2, tmp);
        store_old(sm, tmp);
        fetch_old(z0 - 1, tmp);
        store_old(s0, tmp);
    }
    fetch_old(z0, on);
    fetch_cell(z0 - 2, dm);
    fetch_cell(z0 - 1, dc);
    for (int k = z0 - 1; k <= z1; ++k) {
        // prefetch plane k+1 of my cell and old plane k+2; consumed next step
        fetch_cell(k + 1, dn);
        if (k + 2 <= z1 + 1) fetch_old(k + 2, onn);
        store_old(sp, on);  // old plane k+1
        __syncthreads();
        // ---- first colour on plane k over the tile + 1 halo
        const int gk = axis_cell(k, nz, g.wz);
        {
            T v = T(0);
            if (gk >= 0 && col_ok) {
                const int sy = ty + 1, sx = tx + 1;  // position in the halo-2 arrays
                if ((par ^ (gk & 1)) == first)
                    v = update(ZERO, dc, xo[s0][sy][sx], xo[s0][sy][sx - 1], xo[s0][sy][sx + 1],
                               xo[s0][sy - 1][sx], xo[s0][sy + 1][sx], xo[sm][sy][sx], xo[sp][sy][sx]);
                else
                    v = xo[s0][sy][sx];  // second colour: old value (not used for updates)
            }
            xn[s0][ty][tx] = v;
        }
        __syncthreads();
        // ---- second colour on plane k-1 over the tile; write the tile's plane k-1
        const int kb = k - 1;
        if (kb >= z0 && kb < z1 && interior) {
            T out;
            if ((par ^ (kb & 1)) != first) {
                const T xc = xo[sm][ty + 1][tx + 1];
                out = update(false, dm, xc, xn[sm][ty][tx - 1], xn[sm][ty][tx + 1], xn[sm][ty - 1][tx],
                             xn[sm][ty + 1][tx], xn[sp][ty][tx], xn[s0][ty][tx]);
            } else {
                out = xn[sm][ty][tx];
            }
            xout[kb * plane + col] = out;
        }
        // the next step's store replaces the old plane k-1 read just above
        __syncthreads();
        dm = dc;
        dc = dn;
#pragma unroll
        for (int q = 0; q < NE; ++q) on[q] = onn[q];
        const int t = sm;  // plane k becomes k-1, k+1 becomes k, the slot of k-1 is reused
        sm = s0;
        s0 = sp;
        sp = t;
    }
}

template <typename T>
void launch_rbgs_fused(const Geo& g, const Coef<T>& cf, const T* w, const T* f, const T* xin,
                       T* xout, int first_color, double omega, bool zero_init, bool use_w,
                       cudaStream_t st) {
    dim3 gr((g.nx + FTX - 1) / FTX, (g.ny + FTY - 1) / FTY, (g.nz + FZ - 1) / FZ);
    dim3 bl(HX1, HY1);
    const T om = (T)omega;
    if (zero_init) {
        if (use_w)
            rbgs_fused_kernel<T, true, true><<<gr, bl, 0, st>>>(g, cf, w, f, xin, xout, first_color, om);
        else
            rbgs_fused_kernel<T, true, false><<<gr, bl, 0, st>>>(g, cf, w, f, xin, xout, first_color, om);
    } else {
        if (use_w)
            rbgs_fused_kernel<T, false, true><<<gr, bl, 0, st>>>(g, cf, w, f, xin, xout, first_color, om);
        else
            rbgs_fused_kernel<T, false, false><<<gr, bl, 0, st>>>(g, cf, w, f, xin, xout, first_color, om);
    }
    count_launch();
}

bool rbgs_fused_fits(const Geo& g) {
    const int64_t big = (int64_t)1 << 31;
    return g.nface(0) < big && g.nface(1) < big && g.nface(2) < big;
}

template void launch_rbgs_fused<float>(const Geo&, const Coef<float>&, const float*, const float*,
                                       const float*, float*, int, double, bool, bool, cudaStream_t);
template void launch_rbgs_fused<double>(const Geo&, const Coef<double>&, const double*,
                                        const double*, const double*, double*, int, double, bool,
                                        bool, cudaStream_t);

}  // namespace paris
