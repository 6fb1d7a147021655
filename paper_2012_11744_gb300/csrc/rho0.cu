// Finest-level FP32 operator rebuilt from the cell densities.
//
// In the mixed-precision projection step the FP32 operator of level 0 is
// applied by the colour passes of the smoother, by the residual restriction
// and by the flexible-CG matrix-vector product.  Reading it as three FP32
// face arrays costs 12 bytes per cell and pass; these kernels read one FP32
// array of half-densities rh = rho/2 (Eq. muH, written by the FP64 face
// coefficient kernel, 4 bytes per cell) and rebuild every face coefficient in
// registers as beta_f = 1/(rh_L + rh_R) = 2/(rho_L + rho_R), the coefficient
// the FP64 path stores.  Wall faces have beta = 0 (Sec. 3.8).
//
// Layout: the level-0 FP32 vectors of this mode (the smoother's x and f, the
// inner CG's vectors) are stored colour-split: each row holds its cells of
// colour 0 ((i+j+k) even) in order of i, then those of colour 1.  A colour
// pass then reads and writes the updated colour as one contiguous half-row
// and every neighbour it needs from the other half, instead of moving whole
// rows of which it updates half.  rho/2 stays in cell order.
//
// Thread layout: a thread owns the x-pair of cells (2t, 2t+1) of one row
// (entry t of both half-rows) and walks a segment of z-planes (an even number
// chosen per launch).  The pair's values of the planes above are loaded a few
// planes ahead into a ring of registers, so each warp keeps several planes of
// loads in flight while it computes; the values one plane below are carried
// from the previous step.  The x-neighbours outside the pair are held by the
// adjacent lanes and arrive by warp shuffles (the lanes at the edges of the
// warp load theirs); the y-neighbours are loads of the adjacent rows, mostly
// cache hits.  In a colour pass the updated member of a pair alternates with
// the plane, and since 2t is even the colour of a plane is the same across
// the warp: the loop is unrolled by two planes with the member fixed at
// compile time.
//
// Requirements (rho0_fits): nx, ny, nz even and 32-bit offsets; for the
// restriction a coarse level with every axis halved.
#include "kernels.cuh"

namespace paris {

namespace {

constexpr int kVX = 32;         // pairs per warp: 64 cells along x
constexpr int kWX = 1;          // warps along x per block
constexpr int kVY = 8 / kWX;    // rows per block (8 warps per block)
constexpr int kBX = kVX * kWX;  // threads along x per block
constexpr bool kLockstep = false;  // barrier per plane: a block's warps advance together
constexpr int kPassRing = 4;       // planes in the colour pass's load ring (even)
constexpr unsigned kAll = 0xffffffffu;

__device__ __forceinline__ float rcp_fast(float v) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v));
    return y;
}

// beta of the face between two cells with half-densities a and b
__device__ __forceinline__ float bface(float a, float b) { return rcp_fast(a + b); }

__device__ __forceinline__ float2 ldc2(const float* __restrict__ p, int c) {
    return __ldg(reinterpret_cast<const float2*>(p + c));
}
template <int M>
__device__ __forceinline__ float mem(float2 v) {
    return M ? v.y : v.x;
}

// offset of plane k (wrapped periodically into [0, nz)) plus an in-plane offset
__device__ __forceinline__ int plane_at(int k, int nz, int pl, int in_plane) {
    k = k < 0 ? k + nz : (k >= nz ? k - nz : k);
    return k * pl + in_plane;
}

// Geometry of the pair (2t, 2t+1) of row j shared by the kernels below.
struct PairCtx {
    int nx, ny, nz, pl;
    int cj;              // in-plane offset of cell i0 = 2t (idle lanes shadow the last pair)
    bool act;            // the pair lies in the grid
    bool xm_lane;        // minus neighbour of i0 held by lane-1 (as its .y)
    bool xp_lane;        // plus neighbour of i0+1 held by lane+1 (as its .x)
    bool xm_wall, xp_wall, ym_wall, yp_wall, wz;
    int xm_off, xp_off;  // offsets of those neighbours from cell i0 (periodic wrap)
    int ym, yp;          // offsets of rows j-1, j+1 from row j (periodic wrap)
    // colour-split layout of the FP32 vectors: within a row, the cells of
    // colour 0 ((i+j+k) even) at [0, nx/2), those of colour 1 at [nx/2, nx),
    // each in order of i; pair t holds one cell of each colour, at index t
    int hx;              // nx/2
    int jt;              // j*nx + t: split offset of pair t's colour-0 cell within a plane
    int tm, tp1;         // t-1 and t+1 wrapped around the row (periodic)
    int jpar;            // j & 1: cell i0 of plane k has colour (j + k) & 1
};

__device__ __forceinline__ PairCtx pair_ctx(const Geo& g, int tp, int lane, int j) {
    PairCtx q;
    q.nx = g.nx;
    q.ny = g.ny;
    q.nz = g.nz;
    q.pl = g.nx * g.ny;
    q.act = 2 * tp < g.nx;
    const int i0 = q.act ? 2 * tp : g.nx - 2;
    q.cj = j * g.nx + i0;
    q.xm_lane = lane > 0 && i0 > 0;
    q.xp_lane = lane < kVX - 1 && i0 + 2 < g.nx;
    q.xm_wall = g.wx && i0 == 0;
    q.xp_wall = g.wx && i0 + 2 == g.nx;
    q.xm_off = i0 > 0 ? -1 : g.nx - 1;
    q.xp_off = i0 + 2 < g.nx ? 2 : 2 - g.nx;
    q.ym_wall = g.wy && j == 0;
    q.yp_wall = g.wy && j == g.ny - 1;
    q.ym = j > 0 ? -g.nx : (g.ny - 1) * g.nx;
    q.yp = j < g.ny - 1 ? g.nx : -(g.ny - 1) * g.nx;
    q.wz = g.wz;
    q.hx = g.nx / 2;
    const int t = i0 / 2;
    q.jt = j * g.nx + t;
    q.tm = t > 0 ? -1 : q.hx - 1;
    q.tp1 = t + 1 < q.hx ? 1 : 1 - q.hx;
    q.jpar = j & 1;
    return q;
}

// The x-neighbours outside the pair of a plane (pair values X, R): minus
// side of i0 (.x of the result) and plus side of i0+1 (.y), from the
// adjacent lanes; lanes whose neighbour another warp holds (or that wrap
// around the domain) use the values they loaded ahead (vm, rm / vp, rp).
template <bool MINUS, bool PLUS>
__device__ __forceinline__ void outer_x(const PairCtx& q, float2 X, float2 R, float vm, float rm, float vp,
                                        float rp, float2& vo, float2& ro) {
    if (MINUS) {
        vo.x = __shfl_up_sync(kAll, X.y, 1);
        ro.x = __shfl_up_sync(kAll, R.y, 1);
        if (!q.xm_lane) {
            vo.x = vm;
            ro.x = rm;
        }
    }
    if (PLUS) {
        vo.y = __shfl_down_sync(kAll, X.x, 1);
        ro.y = __shfl_down_sync(kAll, R.x, 1);
        if (!q.xp_lane) {
            vo.y = vp;
            ro.y = rp;
        }
    }
}

inline int pair_blocks_x(const Geo& g) { return (g.nx / 2 + kBX - 1) / kBX; }

__device__ __forceinline__ int pair_index() {
    return (blockIdx.x * kWX + (threadIdx.x >> 5)) * kVX + (threadIdx.x & 31);
}

__device__ __forceinline__ void plane_barrier() {
    if (kLockstep) __syncthreads();
}

// Planes per thread segment: an even number from {2, 4, ..., 32} that
// minimises (full waves of resident blocks) x (planes per segment + 2, the
// planes a segment loads ahead and below), so the last wave is not mostly
// empty and short segments do not repeat too many loads.
int segment_planes(const Geo& g, int nplanes, const void* kernel) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
            cudaGetLastError();
            sms = 1;
        }
    }
    // resident blocks per SM of each kernel (asked once per kernel)
    static const void* keys[8] = {};
    static int vals[8] = {};
    int per_sm = 0;
    for (int e = 0; e < 8 && keys[e]; ++e)
        if (keys[e] == kernel) per_sm = vals[e];
    if (per_sm == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBX * kVY, 0) != cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        for (int e = 0; e < 8; ++e)
            if (!keys[e]) {
                keys[e] = kernel;
                vals[e] = per_sm;
                break;
            }
    }
    const int64_t resident = (int64_t)sms * per_sm;
    const int64_t plane_blocks = (int64_t)pair_blocks_x(g) * ((g.ny + kVY - 1) / kVY);
    int best = 2;
    double best_cost = 1e300;
    for (int seg = 2; seg <= 32; seg += 2) {
        const int64_t nb = plane_blocks * ((nplanes + seg - 1) / seg);
        const double waves = (double)((nb + resident - 1) / resident);
        const double cost = waves * (seg + 2);
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = seg;
        }
    }
    return best;
}

}  // namespace

bool rho0_fits(const Geo& g) {
    if (g.nx % 2 || g.ny % 2 || g.nz % 2) return false;
    const int64_t big = ((int64_t)1 << 31) - 1;
    return g.nface(0) < big && g.nface(1) < big && g.nface(2) < big;
}

// ------------------------------------------------------------ colour pass ---

namespace {

// One plane's values for a colour pass of colour `col` whose updated cell is
// member M of the pair (the other member, of the other colour, is the
// partner).  x and f are in the colour-split layout, rho/2 in cell order.
struct PassSlot {
    float xu, xo;           // x of the updated cell and of the partner
    float2 R;               // rho/2 of the pair (members 0, 1)
    float xym, xyp;         // x of the updated cell's y-neighbours (rows j-1, j+1)
    float rym, ryp;         // and their rho/2
    float f;                // f of the updated cell
    float xe, re;           // x and rho/2 of its x-neighbour outside the pair (edge lanes)
};

template <bool ZERO, int M>
__device__ __forceinline__ void pass_load(PassSlot& s, const PairCtx& q, const float* x,
                                          const float* __restrict__ rh, const float* __restrict__ f,
                                          int col, int k) {
    const int o = plane_at(k, q.nz, q.pl, q.cj);     // cell i0 (rho/2, cell order)
    const int os = plane_at(k, q.nz, q.pl, q.jt);    // pair t, colour 0 (split layout)
    const int ou = os + (col ? q.hx : 0), oo = os + (col ? 0 : q.hx);  // updated / other colour
    s.R = ldc2(rh, o);
    s.rym = __ldg(rh + o + q.ym + M);
    s.ryp = __ldg(rh + o + q.yp + M);
    s.f = __ldg(f + ou);
    // every lane loads the neighbour outside its pair (a valid cell of the
    // same row; only the edge lanes use it): a conditional load would make
    // the selection wait for the load here instead of three planes later
    s.re = __ldg(rh + o + (M == 0 ? q.xm_off : q.xp_off));
    if (ZERO) {
        s.xu = s.xo = s.xym = s.xyp = s.xe = 0.f;
    } else {
        s.xu = x[ou];
        s.xo = x[oo];
        // the updated cell's neighbours all have the other colour
        s.xym = x[oo + q.ym];
        s.xyp = x[oo + q.yp];
        s.xe = x[oo + (M == 0 ? q.tm : q.tp1)];
    }
}

// Over-relaxed Gauss-Seidel update (Eq. eq:beta_pressure, SPD form) of member
// M of the pair in plane k:
//   x_c <- x_c + omega ((h^2 f_c + sum_f beta_f x_nb) / sum_f beta_f - x_c);
// S: this plane, S1: the plane above (its partner is the updated cell's
// z-neighbour), xzm/rzm: x and rho/2 of the z-neighbour below.
template <bool ZERO, int M>
__device__ __forceinline__ void pass_plane(const PairCtx& q, float* x, float h2, float omega, int col, int k,
                                           const PassSlot& S, const PassSlot& S1, float xzm, float rzm) {
    // the x-neighbour outside the pair: the partner of lane -1 (M = 0) or of
    // lane +1 (M = 1); edge lanes use their own loads
    float vo, ro;
    if (M == 0) {
        vo = __shfl_up_sync(kAll, S.xo, 1);
        ro = __shfl_up_sync(kAll, S.R.y, 1);
        if (!q.xm_lane) { vo = S.xe; ro = S.re; }
    } else {
        vo = __shfl_down_sync(kAll, S.xo, 1);
        ro = __shfl_down_sync(kAll, S.R.x, 1);
        if (!q.xp_lane) { vo = S.xe; ro = S.re; }
    }
    const float ru = mem<M>(S.R), rin = mem<1 - M>(S.R);
    const float b0 = (M == 0 ? q.xm_wall : q.xp_wall) ? 0.f : bface(ru, ro);
    const float b1 = bface(ru, rin);
    const float b2 = q.ym_wall ? 0.f : bface(ru, S.rym);
    const float b3 = q.yp_wall ? 0.f : bface(ru, S.ryp);
    const float b4 = (q.wz && k == 0) ? 0.f : bface(ru, rzm);
    const float b5 = (q.wz && k == q.nz - 1) ? 0.f : bface(ru, mem<M>(S1.R));
    const float w = rcp_fast(((b0 + b1) + (b2 + b3)) + (b4 + b5));
    const float fc = S.f * h2;
    float xn;
    if (ZERO) {
        xn = omega * w * fc;
    } else {
        float acc = fmaf(b0, vo, fc);
        acc = fmaf(b1, S.xo, acc);
        acc = fmaf(b2, S.xym, acc);
        acc = fmaf(b3, S.xyp, acc);
        acc = fmaf(b4, xzm, acc);
        acc = fmaf(b5, S1.xo, acc);
        xn = fmaf(omega, fmaf(w, acc, -S.xu), S.xu);
    }
    if (q.act) {
        const int os = k * q.pl + q.jt;
        x[os + (col ? q.hx : 0)] = xn;
        if (ZERO) x[os + (col ? 0 : q.hx)] = 0.f;  // the other colour starts from zero
    }
}

// A ring of R slots over the planes (R even: the updated member alternates
// with the plane).  Step U of a round computes plane k + U from slot U (this
// plane) and slot U+1 (the plane above) after loading plane k + U + R - 1 into
// slot U-1, whose plane (k + U - 1) is done; the round is unrolled, so every
// slot keeps its registers, and the plane above arrives R - 2 steps after its
// load was issued.  A colour pass only reads cells of the other colour and
// the updated cell itself before its update, so loading ahead is safe.
template <bool ZERO, int M0, int R, int U>
struct PassRing {
    __device__ __forceinline__ static bool run(const PairCtx& q, float* x, const float* __restrict__ rh,
                                               const float* __restrict__ f, float h2, float omega, int col,
                                               int k, int ke, PassSlot (&S)[R], float& xzm, float& rzm) {
        constexpr int M = (M0 + U) & 1;  // member updated in plane k + U
        const int kk = k + U;
        if (kk >= ke) return false;
        if (kk + R - 1 <= ke)
            pass_load<ZERO, (M0 + U + R - 1) & 1>(S[(U + R - 1) % R], q, x, rh, f, col, kk + R - 1);
        plane_barrier();
        pass_plane<ZERO, M>(q, x, h2, omega, col, kk, S[U], S[(U + 1) % R], xzm, rzm);
        // the next plane updates the other member; its z-neighbour below is
        // this plane's partner, which this pass does not change
        xzm = S[U].xo;
        rzm = mem<1 - M>(S[U].R);
        return PassRing<ZERO, M0, R, U + 1>::run(q, x, rh, f, h2, omega, col, k, ke, S, xzm, rzm);
    }
};
template <bool ZERO, int M0, int R>
struct PassRing<ZERO, M0, R, R> {
    __device__ __forceinline__ static bool run(const PairCtx&, float*, const float* __restrict__,
                                               const float* __restrict__, float, float, int, int, int,
                                               PassSlot (&)[R], float&, float&) {
        return true;
    }
};

template <bool ZERO, int M0, int R>
__device__ __forceinline__ void pass_loop(const PairCtx& q, float* x, const float* __restrict__ rh,
                                          const float* __restrict__ f, float h2, float omega, int col,
                                          int kb, int ke) {
    static_assert(R % 2 == 0, "the ring length must be even");
    PassSlot S[R];
#pragma unroll
    for (int u = 0; u < R - 1; ++u) {
        if (u % 2 == 0) pass_load<ZERO, M0>(S[u], q, x, rh, f, col, kb + u);
        else pass_load<ZERO, 1 - M0>(S[u], q, x, rh, f, col, kb + u);
    }
    float xzm, rzm;  // the updated cell's z-neighbour below (other colour): x, rho/2
    {
        rzm = __ldg(rh + plane_at(kb - 1, q.nz, q.pl, q.cj) + M0);
        xzm = ZERO ? 0.f : x[plane_at(kb - 1, q.nz, q.pl, q.jt) + (col ? 0 : q.hx)];
    }
    for (int k = kb; k < ke; k += R)
        if (!PassRing<ZERO, M0, R, 0>::run(q, x, rh, f, h2, omega, col, k, ke, S, xzm, rzm)) break;
}

}  // namespace

// ZERO: x is taken as 0 on entry and the other colour is written as 0.
template <bool ZERO>
__global__ void __launch_bounds__(kBX* kVY) rbgs_rho_kernel(Geo g, const float* __restrict__ rh, float h2,
                                                          const float* __restrict__ f,
                                                          float* __restrict__ x, int color,
                                                          float omega, int k0, int k1, int seg) {
    const int j = blockIdx.y * kVY + threadIdx.y;
    const int kb = k0 + blockIdx.z * seg;
    if (kb >= k1) return;  // uniform per block
    if (!kLockstep && j >= g.ny) return;  // uniform per warp
    const int ke = min(kb + seg, k1);
    // rows past the grid (only with the per-plane barrier) shadow the last row
    PairCtx q = pair_ctx(g, pair_index(), threadIdx.x & 31, min(j, g.ny - 1));
    q.act = q.act && j < g.ny;
    // member of the pair updated in plane kb: (i0 + j + kb) has the colour's
    // parity for i0, i0 even
    if (((j + kb + color) & 1) == 0)
        pass_loop<ZERO, 0, kPassRing>(q, x, rh, f, h2, omega, color, kb, ke);
    else
        pass_loop<ZERO, 1, kPassRing>(q, x, rh, f, h2, omega, color, kb, ke);
}

void launch_rbgs_rho(const Geo& g, const float* rh, double h, const float* f, float* x, int color,
                     double omega, bool zero_init, cudaStream_t st, int k0, int k1) {
    if (k1 < 0) k1 = g.nz;
    const float h2 = (float)(h * h);
    if (zero_init) {
        const int seg = segment_planes(g, k1 - k0, (const void*)rbgs_rho_kernel<true>);
        dim3 gr(pair_blocks_x(g), (g.ny + kVY - 1) / kVY, (k1 - k0 + seg - 1) / seg);
        rbgs_rho_kernel<true><<<gr, dim3(kBX, kVY), 0, st>>>(g, rh, h2, f, x, color, (float)omega, k0, k1, seg);
    } else {
        const int seg = segment_planes(g, k1 - k0, (const void*)rbgs_rho_kernel<false>);
        dim3 gr(pair_blocks_x(g), (g.ny + kVY - 1) / kVY, (k1 - k0 + seg - 1) / seg);
        rbgs_rho_kernel<false><<<gr, dim3(kBX, kVY), 0, st>>>(g, rh, h2, f, x, color, (float)omega, k0, k1, seg);
    }
    count_launch();
}

// ------------------------------------------- matvec and residual restriction ---

namespace {

// One plane's values for a full application of A to the pair.  x (or d) and
// f are kept as loaded, as the entries of half-rows 0 and 1 (.x, .y); they
// are put in cell order where they are used, so that no instruction waits
// for a load before the plane that needs it.
struct OpSlot {
    float2 X, R;                // x of the pair (half-rows 0, 1) and rh (cell order)
    float2 Xym, Xyp, Rym, Ryp;  // rows j-1, j+1
    float2 F;                   // restriction: f of the pair (half-rows 0, 1)
    float vm, rm, vp, rp;       // x-neighbours outside the pair (edge lanes)
};

__device__ __forceinline__ float2 ld_halves(const float* __restrict__ x, int os, int hx) {
    return make_float2(__ldg(x + os), __ldg(x + os + hx));
}
// half-row entries (colour 0, colour 1) in cell order; c0: colour of cell i0
__device__ __forceinline__ float2 cell_order(float2 v, int c0) {
    return c0 ? make_float2(v.y, v.x) : v;
}

template <bool WITH_F>
__device__ __forceinline__ void op_load(OpSlot& s, const PairCtx& q, const float* __restrict__ x,
                                        const float* __restrict__ rh, const float* __restrict__ f, int k) {
    const int o = plane_at(k, q.nz, q.pl, q.cj);    // rho/2, cell order
    const int os = plane_at(k, q.nz, q.pl, q.jt);   // x and f, colour-split layout
    const int c0 = (q.jpar + k) & 1;                // colour of cell i0 (nz, ny even)
    s.X = ld_halves(x, os, q.hx);
    s.R = ldc2(rh, o);
    s.Xym = ld_halves(x, os + q.ym, q.hx);
    s.Xyp = ld_halves(x, os + q.yp, q.hx);
    s.Rym = ldc2(rh, o + q.ym);
    s.Ryp = ldc2(rh, o + q.yp);
    if (WITH_F) s.F = ld_halves(f, os, q.hx);
    // unconditional (see pass_load): cell i0-1 has colour 1-c0, cell i0+2 colour c0
    s.vm = __ldg(x + os + (c0 ? 0 : q.hx) + q.tm);
    s.rm = __ldg(rh + o + q.xm_off);
    s.vp = __ldg(x + os + (c0 ? q.hx : 0) + q.tp1);
    s.rp = __ldg(rh + o + q.xp_off);
}

// (A x) / scale for both cells of the pair in plane k: sum_f beta_f (x_c - x_nb)
// in the face order x-, x+, y-, y+, z-, z+ of the face-array operator.
// X: the pair in cell order; Xm: the pair one plane below, Xp: the plane
// above (cell order); Bzm, Bzp: z-faces below and above; c0: colour of cell i0.
__device__ __forceinline__ float2 op_apply(const PairCtx& q, const OpSlot& S, float2 X, int c0, float2 Xm,
                                           float2 Xp, float2 Bzm, float2 Bzp) {
    float2 vo, ro;
    outer_x<true, true>(q, X, S.R, S.vm, S.rm, S.vp, S.rp, vo, ro);
    const float2 Xym = cell_order(S.Xym, c0 ^ 1), Xyp = cell_order(S.Xyp, c0 ^ 1);
    const float bxi = bface(S.R.x, S.R.y);
    const float bxm = q.xm_wall ? 0.f : bface(S.R.x, ro.x);
    const float bxp = q.xp_wall ? 0.f : bface(S.R.y, ro.y);
    const float2 Bym = q.ym_wall ? make_float2(0.f, 0.f)
                                 : make_float2(bface(S.R.x, S.Rym.x), bface(S.R.y, S.Rym.y));
    const float2 Byp = q.yp_wall ? make_float2(0.f, 0.f)
                                 : make_float2(bface(S.R.x, S.Ryp.x), bface(S.R.y, S.Ryp.y));
    float a0 = bxm * (X.x - vo.x);
    a0 = fmaf(bxi, X.x - X.y, a0);
    a0 = fmaf(Bym.x, X.x - Xym.x, a0);
    a0 = fmaf(Byp.x, X.x - Xyp.x, a0);
    a0 = fmaf(Bzm.x, X.x - Xm.x, a0);
    a0 = fmaf(Bzp.x, X.x - Xp.x, a0);
    float a1 = bxi * (X.y - X.x);
    a1 = fmaf(bxp, X.y - vo.y, a1);
    a1 = fmaf(Bym.y, X.y - Xym.y, a1);
    a1 = fmaf(Byp.y, X.y - Xyp.y, a1);
    a1 = fmaf(Bzm.y, X.y - Xm.y, a1);
    a1 = fmaf(Bzp.y, X.y - Xp.y, a1);
    return make_float2(a0, a1);
}

__device__ __forceinline__ float2 zfaces(const PairCtx& q, int k, float2 Rlo, float2 Rhi) {
    // faces between planes k and k+1 (walls at the bottom and top of the domain)
    if (q.wz && (k < 0 || k == q.nz - 1)) return make_float2(0.f, 0.f);
    return make_float2(bface(Rlo.x, Rhi.x), bface(Rlo.y, Rhi.y));
}

}  // namespace

// RESTRICT = false: q = A d and the partial sums of d . q (per thread in FP32,
// across threads and blocks in FP64).
// RESTRICT = true: coarse f = mean over the 2x2x2 children of f - A x on the
// level with every axis halved; the two fine rows of a coarse cell belong to
// the warps 2m and 2m+1 of the block and are added through shared memory.
template <bool RESTRICT>
__global__ void __launch_bounds__(kBX* kVY, 3) op_rho_kernel(Geo g, const float* __restrict__ rh, float ih2,
                                                        const float* __restrict__ x,
                                                        const float* __restrict__ f,
                                                        float* __restrict__ out, Geo cg,
                                                        double* partials, int seg, FinSpec fin) {
    __shared__ float sh[2][kVY][kBX];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int j = blockIdx.y * kVY + ty;
    const bool row_ok = j < g.ny;
    const int jc = row_ok ? j : g.ny - 1;  // idle rows shadow the last row (no stores)
    const int kb = blockIdx.z * seg, ke = min(kb + seg, g.nz);
    const int tp = pair_index();
    const PairCtx q = pair_ctx(g, tp, tx & 31, jc);
    const bool store = row_ok && q.act;
    float loc = 0.f, acc = 0.f;
    // ring of three slots over the planes, unrolled by three so every slot
    // keeps its registers: plane k+2 is loaded into the slot of plane k-1
    // while plane k is computed
    OpSlot A, B, C;
    op_load<RESTRICT>(A, q, x, rh, f, kb);
    op_load<RESTRICT>(B, q, x, rh, f, kb + 1);
    float2 Xm, Bzm;
    {
        Xm = cell_order(ld_halves(x, plane_at(kb - 1, q.nz, q.pl, q.jt), q.hx), (q.jpar + kb - 1) & 1);
        Bzm = zfaces(q, kb - 1, ldc2(rh, plane_at(kb - 1, q.nz, q.pl, q.cj)), A.R);
    }
    int buf = 0;
    auto plane = [&](int k, const OpSlot& S0, const OpSlot& S1) {
        plane_barrier();
        const int c0 = (q.jpar + k) & 1;
        const float2 X = cell_order(S0.X, c0);
        const float2 Bzp = zfaces(q, k, S0.R, S1.R);
        const float2 a = op_apply(q, S0, X, c0, Xm, cell_order(S1.X, c0 ^ 1), Bzm, Bzp);
        if (!RESTRICT) {
            const float2 Q = make_float2(ih2 * a.x, ih2 * a.y);
            if (store) {
                // q in the colour-split layout
                const int os = k * q.pl + q.jt;
                out[os + (c0 ? q.hx : 0)] = Q.x;
                out[os + (c0 ? 0 : q.hx)] = Q.y;
                loc = fmaf(X.x, Q.x, loc);
                loc = fmaf(X.y, Q.y, loc);
            }
        } else {
            const float2 F = cell_order(S0.F, c0);
            acc += (F.x - ih2 * a.x) + (F.y - ih2 * a.y);
            if ((k - kb) & 1) {  // planes 2K, 2K+1 done: add the row pair
                sh[buf][ty][tx] = acc;
                acc = 0.f;
                __syncthreads();
                if ((ty & 1) == 0 && store)
                    out[((k >> 1) * cg.ny + (j >> 1)) * cg.nx + tp] =
                        (sh[buf][ty][tx] + sh[buf][ty + 1][tx]) * 0.125f;
                buf ^= 1;
            }
        }
        Xm = X;
        Bzm = Bzp;
    };
    for (int k = kb; k < ke; k += 3) {
        if (k + 2 <= ke) op_load<RESTRICT>(C, q, x, rh, f, k + 2);
        plane(k, A, B);
        if (k + 1 >= ke) break;
        if (k + 3 <= ke) op_load<RESTRICT>(A, q, x, rh, f, k + 3);
        plane(k + 1, B, C);
        if (k + 2 >= ke) break;
        if (k + 4 <= ke) op_load<RESTRICT>(B, q, x, rh, f, k + 4);
        plane(k + 2, C, A);
    }
    if (!RESTRICT) {
        double red[1] = {(double)loc};
        const int op[1] = {0};
        const int64_t blk = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        block_reduce_store<1>(red, op, partials, blk, ty * kBX + tx);
        finalize_last_block(partials, (int64_t)gridDim.x * gridDim.y * gridDim.z, fin, ty * kBX + tx);
    }
}

int64_t rho0_matvec_blocks(const Geo& g) {
    // the most blocks any segment length (>= 2 planes) gives
    return (int64_t)pair_blocks_x(g) * ((g.ny + kVY - 1) / kVY) * ((g.nz + 1) / 2);
}

int64_t launch_matvec_rho(const Geo& g, const float* rh, double h, const float* d, float* q,
                          double* partials, cudaStream_t st, FinSpec fin) {
    const int seg = segment_planes(g, g.nz, (const void*)op_rho_kernel<false>);
    dim3 gr(pair_blocks_x(g), (g.ny + kVY - 1) / kVY, (g.nz + seg - 1) / seg);
    op_rho_kernel<false><<<gr, dim3(kBX, kVY), 0, st>>>(g, rh, (float)(1.0 / (h * h)), d, nullptr, q, g,
                                                        partials, seg, fin);
    count_launch();
    return (int64_t)gr.x * gr.y * gr.z;
}

void launch_restrict_rho(const Geo& g, const float* rh, double h, const float* f, const float* x,
                         const Geo& cg, float* fc, cudaStream_t st) {
    const int seg = segment_planes(g, g.nz, (const void*)op_rho_kernel<true>);
    dim3 gr(pair_blocks_x(g), (g.ny + kVY - 1) / kVY, (g.nz + seg - 1) / seg);
    op_rho_kernel<true><<<gr, dim3(kBX, kVY), 0, st>>>(g, rh, (float)(1.0 / (h * h)), x, f, fc, cg,
                                                       nullptr, seg, no_fin());
    count_launch();
}

// ---------------------------------------------------------- prolongation ---

// x += P xc onto a colour-split finest level from the level with every axis
// halved (piecewise-constant P): entry t of both half-rows of row (j, k) is a
// child of coarse cell (t, j/2, k/2).  V = 4: four entries per thread.
template <int V>
__global__ void prolong_split_kernel(Geo fg, Geo cg, const float* __restrict__ xc, float* __restrict__ x) {
    const int hx = fg.nx / 2;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (t >= hx || j >= fg.ny) return;
    const int rb = (k * fg.ny + j) * fg.nx + t;
    const int cb = ((k >> 1) * cg.ny + (j >> 1)) * cg.nx + t;
    if (V == 4) {
        const float4 a = *reinterpret_cast<const float4*>(xc + cb);
        float4 u = *reinterpret_cast<const float4*>(x + rb);
        float4 w = *reinterpret_cast<const float4*>(x + rb + hx);
        u.x += a.x; u.y += a.y; u.z += a.z; u.w += a.w;
        w.x += a.x; w.y += a.y; w.z += a.z; w.w += a.w;
        *reinterpret_cast<float4*>(x + rb) = u;
        *reinterpret_cast<float4*>(x + rb + hx) = w;
    } else {
        const float a = xc[cb];
        x[rb] += a;
        x[rb + hx] += a;
    }
}

void launch_prolong_split(const Geo& fine, const Geo& coarse, const float* xc, float* x, cudaStream_t st) {
    const int hx = fine.nx / 2;
    const bool v4 = hx % 4 == 0 && ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(xc)) & 15) == 0;
    const int per = v4 ? 4 : 1;
    dim3 blk(32, 8);
    dim3 gr((hx / per + 31) / 32, (fine.ny + 7) / 8, fine.nz);
    if (v4) prolong_split_kernel<4><<<gr, blk, 0, st>>>(fine, coarse, xc, x);
    else prolong_split_kernel<1><<<gr, blk, 0, st>>>(fine, coarse, xc, x);
    count_launch();
}

// --------------------------------------------------- level-1 coefficients ---

// beta of the level with every axis halved: the mean of the four fine faces
// that tile each coarse face, times (h0/h1)^2 = 1/4 and the fine scale
// 1/h0^2 (the coarse arrays hold scaled coefficients).
template <int AXIS>
__global__ void coarse_beta_rho_kernel(Geo fg, const float* __restrict__ rh, float scale, Geo cg,
                                       float* __restrict__ out) {
    const int n0 = cg.nx + (AXIS == 0 ? cg.wx : 0);
    const int n1 = cg.ny + (AXIS == 1 ? cg.wy : 0);
    const int n2 = cg.nz + (AXIS == 2 ? cg.wz : 0);
    const int total = n0 * n1 * n2;
    const int wall = AXIS == 0 ? fg.wx : (AXIS == 1 ? fg.wy : fg.wz);
    const int fn = AXIS == 0 ? fg.nx : (AXIS == 1 ? fg.ny : fg.nz);
    const int cn = AXIS == 0 ? cg.nx : (AXIS == 1 ? cg.ny : cg.nz);
    const int stride = AXIS == 0 ? 1 : (AXIS == 1 ? fg.nx : fg.nx * fg.ny);  // fine cell step along AXIS
    // fine steps along the two other axes
    const int sb = AXIS == 0 ? fg.nx : 1;
    const int se = AXIS == 2 ? fg.nx : fg.nx * fg.ny;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int I = t % n0, J = (t / n0) % n1, K = t / (n0 * n1);
        const int F = AXIS == 0 ? I : (AXIS == 1 ? J : K);
        if (wall && (F == 0 || F == cn)) {
            out[t] = 0.f;
            continue;
        }
        // fine cells on either side of the face plane 2F along AXIS; the
        // corner cell of the four fine faces along the other axes
        const int lo = (2 * F - 1 + fn) % fn, hi = 2 * F;
        const int i = 2 * I, jj = 2 * J, k = 2 * K;
        int base = (k * fg.ny + jj) * fg.nx + i;  // fine cell (2I, 2J, 2K)
        base += (lo - 2 * F) * stride;            // move to plane lo along AXIS (wraps for F = 0)
        const int dhi = (hi - lo) * stride;
        float s = 0.f;
        for (int de = 0; de < 2; ++de)
            for (int db = 0; db < 2; ++db) {
                const int cl = base + db * sb + de * se;
                s += bface(__ldg(rh + cl), __ldg(rh + cl + dhi));
            }
        out[t] = s * scale;
    }
}

void launch_coarse_beta_rho(const Geo& fine, const float* rh, double h, const Geo& coarse, float* out[3],
                            cudaStream_t st) {
    // mean of 4 faces (1/4) x (h0/h1)^2 (1/4) x 1/h0^2
    const float scale = (float)(1.0 / (16.0 * h * h));
    coarse_beta_rho_kernel<0><<<elementwise_blocks(coarse.nface(0)), kRedThreads, 0, st>>>(fine, rh, scale, coarse, out[0]);
    coarse_beta_rho_kernel<1><<<elementwise_blocks(coarse.nface(1)), kRedThreads, 0, st>>>(fine, rh, scale, coarse, out[1]);
    coarse_beta_rho_kernel<2><<<elementwise_blocks(coarse.nface(2)), kRedThreads, 0, st>>>(fine, rh, scale, coarse, out[2]);
    count_launch(3);
}

}  // namespace paris
