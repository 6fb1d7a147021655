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
// Two kernel families apply the operator.  Where nx/2 is even, the
// plane-tile kernels (rbgs_rho_tile_kernel, op_rho_tile_kernel, below) give a
// thread two consecutive pairs of one row of one plane and read every
// half-row as a vector; blocks sweep the planes in order, so the planes above
// and below come from L2.  They stream the level faster and are the ones the
// projection step uses.  The z-column kernels described next serve odd nx/2
// (and paris_opts.level0_tiles = 0).
//
// Z-column thread layout: a thread owns the x-pair of cells (2t, 2t+1) of one
// row (entry t of both half-rows) and walks a segment of z-planes (an even
// number chosen per launch).  The pair's values of the planes above are loaded a few
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

#include <type_traits>

namespace paris {

namespace {

constexpr int kVX = 32;         // pairs per warp: 64 cells along x
constexpr int kWX = 1;          // warps along x per block
constexpr int kVY = 8 / kWX;    // rows per block (8 warps per block)
constexpr int kBX = kVX * kWX;  // threads along x per block
constexpr bool kLockstep = false;  // barrier per plane: a block's warps advance together
constexpr int kPassRing = 4;       // planes in the colour pass's load ring (even)
constexpr int kTileV = 2;          // pairs per lane of the plane-tile colour pass (0: the ring kernel only)
constexpr int kTileOpV = 2;        // pairs per lane of the plane-tile product and restriction (0: ring)
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
// with the plane).  Step U of a turn of the ring computes plane k + U from
// slot U (this plane) and slot U+1 (the plane above) after loading plane
// k + U + R - 1 into slot U-1, whose plane (k + U - 1) is done; the turn is
// unrolled, so every slot keeps its registers, and the plane above arrives
// R - 2 steps after its load was issued.  A colour pass only reads cells of the other colour and
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

// ---- the colour pass over plane tiles, V pairs per lane
//
// A block updates one colour in an 8-row tile of one plane; blocks are
// ordered plane by plane, so the GPU sweeps each array through z as a whole
// and the planes above and below a tile (read again by the tiles of those
// planes) come from L2.  Each lane owns V consecutive pairs of a row: its
// loads are V-wide vectors of the half-rows (16 bytes for V = 4), which
// streams the level faster than one pair per lane with any depth of
// prefetch.  Same update, in the same arithmetic order, as pass_plane.

namespace {

template <int N>
__device__ __forceinline__ void ldv(float (&d)[N], const float* p) {
    static_assert(N == 2 || N == 4 || N == 8, "vector of 2, 4 or 8 floats");
    if constexpr (N == 2) {
        const float2 a = *reinterpret_cast<const float2*>(p);
        d[0] = a.x;
        d[1] = a.y;
    } else {
#pragma unroll
        for (int h = 0; h < N / 4; ++h) {
            const float4 a = *reinterpret_cast<const float4*>(p + 4 * h);
            d[4 * h] = a.x;
            d[4 * h + 1] = a.y;
            d[4 * h + 2] = a.z;
            d[4 * h + 3] = a.w;
        }
    }
}
template <int N>
__device__ __forceinline__ void ldgv(float (&d)[N], const float* __restrict__ p) {
    static_assert(N == 2 || N == 4 || N == 8, "vector of 2, 4 or 8 floats");
    if constexpr (N == 2) {
        const float2 a = __ldg(reinterpret_cast<const float2*>(p));
        d[0] = a.x;
        d[1] = a.y;
    } else {
#pragma unroll
        for (int h = 0; h < N / 4; ++h) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(p + 4 * h));
            d[4 * h] = a.x;
            d[4 * h + 1] = a.y;
            d[4 * h + 2] = a.z;
            d[4 * h + 3] = a.w;
        }
    }
}
// N FP16 values widened to FP32 (N = 4: one 8-byte load, aligned to 8 bytes)
template <int N>
__device__ __forceinline__ void ldgv(float (&d)[N], const __half* __restrict__ p) {
    static_assert(N == 2 || N == 4 || N == 8, "vector of 2, 4 or 8 halves");
    if constexpr (N == 2) {
        const float2 a = __half22float2(__ldg(reinterpret_cast<const __half2*>(p)));
        d[0] = a.x;
        d[1] = a.y;
    } else {
#pragma unroll
        for (int h = 0; h < N / 4; ++h) {
            const uint2 raw = __ldg(reinterpret_cast<const uint2*>(p + 4 * h));
            const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&raw.x));
            const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&raw.y));
            d[4 * h] = a.x;
            d[4 * h + 1] = a.y;
            d[4 * h + 2] = b.x;
            d[4 * h + 3] = b.y;
        }
    }
}
__device__ __forceinline__ float ldr(const float* __restrict__ p) { return __ldg(p); }
__device__ __forceinline__ float ldr(const __half* __restrict__ p) { return __half2float(__ldg(p)); }

template <int N>
__device__ __forceinline__ void stv(float* p, const float (&d)[N]) {
    if constexpr (N == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(d[0], d[1]);
    } else {
        *reinterpret_cast<float4*>(p) = make_float4(d[0], d[1], d[2], d[3]);
    }
}

// member M of the V pairs (2t0 + 2v + M) is updated; walls as in pass_plane.
// ZERO: x is taken as 0 everywhere (nothing of x is read) and only the
// updated colour is written; XZ: the updated colour is taken as 0 (the pass
// after a ZERO pass of the other colour, which left it unwritten).
template <bool ZERO, bool XZ, int V, int M, typename RT>
__device__ __forceinline__ void tile_update(const Geo& g, const RT* __restrict__ rh,
                                            const float* __restrict__ f, float* x, float h2, float omega,
                                            int col, int j, int k, int t0, int lane, bool act) {
    const int nx = g.nx, hx = nx / 2, pl = nx * g.ny;
    const int rb = k * pl + j * nx;
    const int su = rb + (col ? hx : 0) + t0;  // updated colour, entries t0 .. t0+V-1
    const int so = rb + (col ? 0 : hx) + t0;  // the other colour
    const int o = rb + 2 * t0;                // rho/2 of cells 2t0 .. 2t0+2V-1
    const int ym = j > 0 ? -nx : (g.ny - 1) * nx, yp = j < g.ny - 1 ? nx : -(g.ny - 1) * nx;
    const int zm = k > 0 ? -pl : (g.nz - 1) * pl, zp = k < g.nz - 1 ? pl : -(g.nz - 1) * pl;
    float R[2 * V], F[V], Q[2 * V];
    float rym[V], ryp[V], rzm[V], rzp[V];
    ldgv<2 * V>(R, rh + o);
    ldgv<V>(F, f + su);
    ldgv<2 * V>(Q, rh + o + ym);
#pragma unroll
    for (int v = 0; v < V; ++v) rym[v] = Q[2 * v + M];
    ldgv<2 * V>(Q, rh + o + yp);
#pragma unroll
    for (int v = 0; v < V; ++v) ryp[v] = Q[2 * v + M];
    ldgv<2 * V>(Q, rh + o + zm);
#pragma unroll
    for (int v = 0; v < V; ++v) rzm[v] = Q[2 * v + M];
    ldgv<2 * V>(Q, rh + o + zp);
#pragma unroll
    for (int v = 0; v < V; ++v) rzp[v] = Q[2 * v + M];
    // the x-neighbour outside the lane's entries: cell 2t0-1 (M = 0) or
    // 2t0+2V (M = 1), of the other colour, wrapped around the row
    const int te = M == 0 ? (t0 > 0 ? -1 : hx - 1) : (t0 + V < hx ? V : V - hx);
    const float re = ldr(rh + o + (M == 0 ? (t0 > 0 ? -1 : nx - 1) : (t0 + V < hx ? 2 * V : 2 * V - nx)));
    float xu[V], xo[V], xym[V], xyp[V], xzm[V], xzp[V], xe = 0.f;
    if (ZERO) {
#pragma unroll
        for (int v = 0; v < V; ++v) xu[v] = xo[v] = xym[v] = xyp[v] = xzm[v] = xzp[v] = 0.f;
    } else {
        if (XZ) {
#pragma unroll
            for (int v = 0; v < V; ++v) xu[v] = 0.f;
        } else {
            ldv<V>(xu, x + su);
        }
        ldv<V>(xo, x + so);
        ldv<V>(xym, x + so + ym);
        ldv<V>(xyp, x + so + yp);
        ldv<V>(xzm, x + so + zm);
        ldv<V>(xzp, x + so + zp);
        xe = x[so + te];
    }
    // neighbours outside the pair: within the lane's entries, from the
    // adjacent lane, or (lane at the edge of the warp or of the row) loaded
    float vo[V], ro[V];
    if (M == 0) {
        const float px = __shfl_up_sync(kAll, xo[V - 1], 1), pr = __shfl_up_sync(kAll, R[2 * V - 1], 1);
        const bool from_lane = lane > 0 && t0 > 0;
        vo[0] = from_lane ? px : xe;
        ro[0] = from_lane ? pr : re;
#pragma unroll
        for (int v = 1; v < V; ++v) {
            vo[v] = xo[v - 1];
            ro[v] = R[2 * v - 1];
        }
    } else {
        const float nxv = __shfl_down_sync(kAll, xo[0], 1), nr = __shfl_down_sync(kAll, R[0], 1);
        const bool from_lane = lane < 31 && t0 + V < hx;
#pragma unroll
        for (int v = 0; v < V - 1; ++v) {
            vo[v] = xo[v + 1];
            ro[v] = R[2 * v + 2];
        }
        vo[V - 1] = from_lane ? nxv : xe;
        ro[V - 1] = from_lane ? nr : re;
    }
    const bool ym_wall = g.wy && j == 0, yp_wall = g.wy && j == g.ny - 1;
    const bool zm_wall = g.wz && k == 0, zp_wall = g.wz && k == g.nz - 1;
    float xn[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const bool xwall = g.wx && (M == 0 ? (t0 + v == 0) : (t0 + v == hx - 1));
        const float ru = R[2 * v + M], rin = R[2 * v + 1 - M];
        const float b0 = xwall ? 0.f : bface(ru, ro[v]);
        const float b1 = bface(ru, rin);
        const float b2 = ym_wall ? 0.f : bface(ru, rym[v]);
        const float b3 = yp_wall ? 0.f : bface(ru, ryp[v]);
        const float b4 = zm_wall ? 0.f : bface(ru, rzm[v]);
        const float b5 = zp_wall ? 0.f : bface(ru, rzp[v]);
        const float w = rcp_fast(((b0 + b1) + (b2 + b3)) + (b4 + b5));
        const float fc = F[v] * h2;
        if (ZERO) {
            xn[v] = omega * w * fc;
        } else {
            float acc = fmaf(b0, vo[v], fc);
            acc = fmaf(b1, xo[v], acc);
            acc = fmaf(b2, xym[v], acc);
            acc = fmaf(b3, xyp[v], acc);
            acc = fmaf(b4, xzm[v], acc);
            acc = fmaf(b5, xzp[v], acc);
            xn[v] = fmaf(omega, fmaf(w, acc, -xu[v]), xu[v]);
        }
    }
    if (act) stv<V>(x + su, xn);
}

// The regular colour pass (x read) on two consecutive planes k and k+1 of
// row j: plane k updates member M of its pairs, plane k+1 member 1 - M.  The
// rows the two share are loaded once: rho/2 of row j in both planes (each
// plane's z-neighbour row is the other's centre row) and x of the other
// colour in both planes (plane k's x above is plane k+1's other colour, and
// plane k+1's x below is plane k's).  Each cell's update is that of
// tile_update, faces in the same order.
template <bool ZERO, bool XZ, int V, int M, typename RT>
__device__ __forceinline__ void tile_update2(const Geo& g, const RT* __restrict__ rh,
                                             const float* __restrict__ f, float* x, float h2, float omega,
                                             int col, int j, int k, int t0, int lane, bool act) {
    const int nx = g.nx, hx = nx / 2, pl = nx * g.ny;
    const int rb = k * pl + j * nx;
    const int su = rb + (col ? hx : 0) + t0;  // updated colour of plane k (plane k+1: + pl)
    const int so = rb + (col ? 0 : hx) + t0;  // the other colour of plane k (plane k+1: + pl)
    const int o = rb + 2 * t0;                // rho/2 of cells 2t0 .. 2t0+2V-1 of plane k (k+1: + pl)
    const int ym = j > 0 ? -nx : (g.ny - 1) * nx, yp = j < g.ny - 1 ? nx : -(g.ny - 1) * nx;
    const int zm = k > 0 ? -pl : (g.nz - 1) * pl;                      // below plane k
    const int zp1 = k + 1 < g.nz - 1 ? pl : -(g.nz - 1) * pl;          // above plane k+1
    float R0[2 * V], R1[2 * V], Q[2 * V];
    ldgv<2 * V>(R0, rh + o);
    ldgv<2 * V>(R1, rh + o + pl);
    float F0[V], F1[V];
    ldgv<V>(F0, f + su);
    ldgv<V>(F1, f + su + pl);
    float rym0[V], ryp0[V], rzm0[V], rym1[V], ryp1[V], rzp1[V];
    ldgv<2 * V>(Q, rh + o + ym);
#pragma unroll
    for (int v = 0; v < V; ++v) rym0[v] = Q[2 * v + M];
    ldgv<2 * V>(Q, rh + o + yp);
#pragma unroll
    for (int v = 0; v < V; ++v) ryp0[v] = Q[2 * v + M];
    ldgv<2 * V>(Q, rh + o + zm);
#pragma unroll
    for (int v = 0; v < V; ++v) rzm0[v] = Q[2 * v + M];
    ldgv<2 * V>(Q, rh + o + pl + ym);
#pragma unroll
    for (int v = 0; v < V; ++v) rym1[v] = Q[2 * v + 1 - M];
    ldgv<2 * V>(Q, rh + o + pl + yp);
#pragma unroll
    for (int v = 0; v < V; ++v) ryp1[v] = Q[2 * v + 1 - M];
    ldgv<2 * V>(Q, rh + o + pl + zp1);
#pragma unroll
    for (int v = 0; v < V; ++v) rzp1[v] = Q[2 * v + 1 - M];
    // edge neighbours (plane k: member M's side; plane k+1: the other side)
    const int teL = t0 > 0 ? -1 : hx - 1, teR = t0 + V < hx ? V : V - hx;
    const int reL = t0 > 0 ? -1 : nx - 1, reR = t0 + V < hx ? 2 * V : 2 * V - nx;
    const float re0 = ldr(rh + o + (M == 0 ? reL : reR));
    const float re1 = ldr(rh + o + pl + (M == 0 ? reR : reL));
    float xu0[V], xo0[V], xym0[V], xyp0[V], xzm0[V];
    float xu1[V], xo1[V], xym1[V], xyp1[V], xzp1[V];
    float xe0 = 0.f, xe1 = 0.f;
    if (ZERO) {
#pragma unroll
        for (int v = 0; v < V; ++v)
            xu0[v] = xo0[v] = xym0[v] = xyp0[v] = xzm0[v] = xu1[v] = xo1[v] = xym1[v] = xyp1[v] = xzp1[v] = 0.f;
    } else {
        if (XZ) {
#pragma unroll
            for (int v = 0; v < V; ++v) xu0[v] = xu1[v] = 0.f;
        } else {
            ldv<V>(xu0, x + su);
            ldv<V>(xu1, x + su + pl);
        }
        ldv<V>(xo0, x + so);
        ldv<V>(xym0, x + so + ym);
        ldv<V>(xyp0, x + so + yp);
        ldv<V>(xzm0, x + so + zm);
        ldv<V>(xo1, x + so + pl);
        ldv<V>(xym1, x + so + pl + ym);
        ldv<V>(xyp1, x + so + pl + yp);
        ldv<V>(xzp1, x + so + pl + zp1);
        xe0 = x[so + (M == 0 ? teL : teR)];
        xe1 = x[so + pl + (M == 0 ? teR : teL)];
    }
    const bool ym_wall = g.wy && j == 0, yp_wall = g.wy && j == g.ny - 1;
    const bool zm_wall = g.wz && k == 0, zp_wall = g.wz && k + 1 == g.nz - 1;
    // one plane's update: member MM, its rows and neighbours; rzm / xzm the
    // plane below, rzp / xzp the plane above (the other plane's rows where
    // they are shared)
    auto update = [&](auto mm, const float (&R)[2 * V], const float (&F)[V], const float (&rym)[V],
                      const float (&ryp)[V], const float (&rzm)[V], const float (&rzp)[V], const float (&xu)[V],
                      const float (&xo)[V], const float (&xym)[V], const float (&xyp)[V], const float (&xzm)[V],
                      const float (&xzp)[V], float xe, float re, bool zmw, bool zpw, float (&xn)[V]) {
        constexpr int MM = decltype(mm)::value;
        float vo[V], ro[V];
        if (MM == 0) {
            const float px = __shfl_up_sync(kAll, xo[V - 1], 1), pr = __shfl_up_sync(kAll, R[2 * V - 1], 1);
            const bool from_lane = lane > 0 && t0 > 0;
            vo[0] = from_lane ? px : xe;
            ro[0] = from_lane ? pr : re;
#pragma unroll
            for (int v = 1; v < V; ++v) {
                vo[v] = xo[v - 1];
                ro[v] = R[2 * v - 1];
            }
        } else {
            const float nxv = __shfl_down_sync(kAll, xo[0], 1), nr = __shfl_down_sync(kAll, R[0], 1);
            const bool from_lane = lane < 31 && t0 + V < hx;
#pragma unroll
            for (int v = 0; v < V - 1; ++v) {
                vo[v] = xo[v + 1];
                ro[v] = R[2 * v + 2];
            }
            vo[V - 1] = from_lane ? nxv : xe;
            ro[V - 1] = from_lane ? nr : re;
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const bool xwall = g.wx && (MM == 0 ? (t0 + v == 0) : (t0 + v == hx - 1));
            const float ru = R[2 * v + MM], rin = R[2 * v + 1 - MM];
            const float b0 = xwall ? 0.f : bface(ru, ro[v]);
            const float b1 = bface(ru, rin);
            const float b2 = ym_wall ? 0.f : bface(ru, rym[v]);
            const float b3 = yp_wall ? 0.f : bface(ru, ryp[v]);
            const float b4 = zmw ? 0.f : bface(ru, rzm[v]);
            const float b5 = zpw ? 0.f : bface(ru, rzp[v]);
            const float w = rcp_fast(((b0 + b1) + (b2 + b3)) + (b4 + b5));
            const float fc = F[v] * h2;
            if (ZERO) {
                xn[v] = omega * w * fc;
            } else {
                float acc = fmaf(b0, vo[v], fc);
                acc = fmaf(b1, xo[v], acc);
                acc = fmaf(b2, xym[v], acc);
                acc = fmaf(b3, xyp[v], acc);
                acc = fmaf(b4, xzm[v], acc);
                acc = fmaf(b5, xzp[v], acc);
                xn[v] = fmaf(omega, fmaf(w, acc, -xu[v]), xu[v]);
            }
        }
    };
    // plane k: above it plane k+1's row (rho/2 of member M, x of the other colour of plane k+1)
    float rzp0[V], rzm1[V], xn0[V], xn1[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        rzp0[v] = R1[2 * v + M];
        rzm1[v] = R0[2 * v + 1 - M];
    }
    update(std::integral_constant<int, M>{}, R0, F0, rym0, ryp0, rzm0, rzp0, xu0, xo0, xym0, xyp0, xzm0, xo1, xe0,
           re0, zm_wall, false, xn0);
    update(std::integral_constant<int, 1 - M>{}, R1, F1, rym1, ryp1, rzm1, rzp1, xu1, xo1, xym1, xyp1, xo0, xzp1,
           xe1, re1, false, zp_wall, xn1);
    if (act) {
        stv<V>(x + su, xn0);
        stv<V>(x + su + pl, xn1);
    }
}

}  // namespace

#ifndef PARIS_TILE_MINB
#define PARIS_TILE_MINB 1
#endif
// with rho/2 in FP16 the pass is closer to issue-bound: six blocks per SM
// (40 registers) measured 2 % faster than the register-unbounded five
#ifndef PARIS_TILE_MINB_H
#define PARIS_TILE_MINB_H 6
#endif
// the regular pass of the V-cycle on two planes per block (1: one plane per block)
#ifndef PARIS_TILE_NP
#define PARIS_TILE_NP 2
#endif
// rows per block of the two-plane pass: blocks of two rows (64 threads, 16
// per SM at 64 registers) measured 28.6 us a pass against 30.3 with eight
// rows and 32.4 with sixteen
#ifndef PARIS_TILE2_VY
#define PARIS_TILE2_VY 2
#endif
constexpr int kVY2 = PARIS_TILE2_VY;
#ifndef PARIS_TILE2_MINB
#define PARIS_TILE2_MINB (32 / PARIS_TILE2_VY)
#endif
// the zero-initial pass and the pass after it on two planes per block
#ifndef PARIS_TILE_NP_ZERO
#define PARIS_TILE_NP_ZERO 2
#endif
#ifndef PARIS_TILE_NP_XZ
#define PARIS_TILE_NP_XZ 2
#endif
template <bool ZERO, bool XZ, int V, typename RT = float>
__global__ void __launch_bounds__(kBX* kVY, sizeof(RT) == 2 ? PARIS_TILE_MINB_H : PARIS_TILE_MINB) rbgs_rho_tile_kernel(Geo g, const RT* __restrict__ rh, float h2,
                                                               const float* __restrict__ f, float* x,
                                                               int color, float omega, int k0, int rev) {
    pdl_wait();
    const int j = blockIdx.y * kVY + threadIdx.y;
    if (j >= g.ny) return;  // uniform per warp
    // rev: the planes in descending order (the blocks of a grid start in
    // ascending blockIdx order, so a pass that runs against the previous one
    // begins where that one ended, on planes still in L2; the cells of one
    // colour are independent, so the order changes no value)
    const int k = k0 + (rev ? (int)(gridDim.z - 1 - blockIdx.z) : (int)blockIdx.z);
    const int lane = threadIdx.x & 31;
    const int hx = g.nx / 2;
    const int tv = (blockIdx.x * kBX + threadIdx.x) * V;
    const bool act = tv < hx;
    const int t0 = act ? tv : hx - V;  // idle lanes shadow the last entries (no stores)
    // cell 2t0 has colour (j + k) & 1: the updated member is the same for the whole row
    if (((j + k + color) & 1) == 0)
        tile_update<ZERO, XZ, V, 0, RT>(g, rh, f, x, h2, omega, color, j, k, t0, lane, act);
    else
        tile_update<ZERO, XZ, V, 1, RT>(g, rh, f, x, h2, omega, color, j, k, t0, lane, act);
}

// The colour pass over pairs of planes (tile_update2; ZERO, XZ as in
// tile_update): block z covers planes k0 + 2 zb and k0 + 2 zb + 1 (rev: zb
// descending).
template <bool ZERO, bool XZ, int V, typename RT>
__global__ void __launch_bounds__(kBX* kVY2, PARIS_TILE2_MINB) rbgs_rho_tile2_kernel(Geo g, const RT* __restrict__ rh,
                                                                                   float h2, const float* __restrict__ f,
                                                                                   float* x, int color, float omega,
                                                                                   int k0, int rev) {
    pdl_wait();
    const int j = blockIdx.y * kVY2 + threadIdx.y;
    if (j >= g.ny) return;  // uniform per warp
    const int zb = rev ? (int)(gridDim.z - 1 - blockIdx.z) : (int)blockIdx.z;
    const int k = k0 + 2 * zb;
    const int lane = threadIdx.x & 31;
    const int hx = g.nx / 2;
    const int tv = (blockIdx.x * kBX + threadIdx.x) * V;
    const bool act = tv < hx;
    const int t0 = act ? tv : hx - V;  // idle lanes shadow the last entries (no stores)
    if (((j + k + color) & 1) == 0)
        tile_update2<ZERO, XZ, V, 0, RT>(g, rh, f, x, h2, omega, color, j, k, t0, lane, act);
    else
        tile_update2<ZERO, XZ, V, 1, RT>(g, rh, f, x, h2, omega, color, j, k, t0, lane, act);
}

bool rho0_tile_pass(const Geo& g, int tiles) {
    return (tiles == 2 && rho0_stage_fits(g)) || (tiles != 0 && kTileV > 0 && (g.nx / 2) % kTileV == 0);
}

void launch_rbgs_rho(const Geo& g, const float* rh, double h, const float* f, float* x, int color,
                     double omega, bool zero_init, cudaStream_t st, int k0, int k1, int tiles, bool own_zero,
                     unsigned* fail, const __half* rh16, bool rev) {
    if (k1 < 0) k1 = g.nz;
    const bool al16 = (((uintptr_t)rh | (uintptr_t)f | (uintptr_t)x) & 15u) == 0;  // bulk copies: 16-byte aligned
    if (tiles == 2 && fail && al16 && rho0_stage_fits(g)) {
        const cudaError_t e = launch_rbgs_rho_stage(g, rh, h, f, x, color, omega, zero_init, own_zero, k0, k1, fail, st);
        if (e != cudaSuccess) paris_internal_note_cuda_error(e);
        return;
    }
    const float h2 = (float)(h * h);
    const int hx = g.nx / 2;
    if (tiles != 0 && kTileV > 0 && (g.nx / 2) % kTileV == 0) {
        constexpr int V = kTileV > 0 ? kTileV : 2;
        dim3 gr((hx / V + kBX - 1) / kBX, (g.ny + kVY - 1) / kVY, k1 - k0);
        if (rh16 && tiles == 1) {  // the V-cycle's passes from FP16 rho/2
            const dim3 gr2(gr.x, (g.ny + kVY2 - 1) / kVY2, (k1 - k0) / 2);
            const bool two = (k1 - k0) % 2 == 0;
            if (zero_init && two && PARIS_TILE_NP_ZERO == 2)
                launch_pdl(rbgs_rho_tile2_kernel<true, false, V, __half>, gr2, dim3(kBX, kVY2), 0, st, g, rh16, h2, f,
                           x, color, (float)omega, k0, rev ? 1 : 0);
            else if (zero_init)
                launch_pdl(rbgs_rho_tile_kernel<true, false, V, __half>, gr, dim3(kBX, kVY), 0, st, g, rh16, h2, f,
                           x, color, (float)omega, k0, rev ? 1 : 0);
            else if (own_zero && two && PARIS_TILE_NP_XZ == 2)
                launch_pdl(rbgs_rho_tile2_kernel<false, true, V, __half>, gr2, dim3(kBX, kVY2), 0, st, g, rh16, h2, f,
                           x, color, (float)omega, k0, rev ? 1 : 0);
            else if (own_zero)
                launch_pdl(rbgs_rho_tile_kernel<false, true, V, __half>, gr, dim3(kBX, kVY), 0, st, g, rh16, h2, f,
                           x, color, (float)omega, k0, rev ? 1 : 0);
            else if (PARIS_TILE_NP == 2 && two)
                launch_pdl(rbgs_rho_tile2_kernel<false, false, V, __half>, gr2, dim3(kBX, kVY2), 0, st, g, rh16, h2, f,
                           x, color, (float)omega, k0, rev ? 1 : 0);
            else
                launch_pdl(rbgs_rho_tile_kernel<false, false, V, __half>, gr, dim3(kBX, kVY), 0, st, g, rh16, h2, f,
                           x, color, (float)omega, k0, rev ? 1 : 0);
            count_launch();
            return;
        }
        if (zero_init)
            launch_pdl(rbgs_rho_tile_kernel<true, false, V>, gr, dim3(kBX, kVY), 0, st, g, rh, h2, f, x, color,
                (float)omega, k0, rev ? 1 : 0);
        else if (own_zero)
            launch_pdl(rbgs_rho_tile_kernel<false, true, V>, gr, dim3(kBX, kVY), 0, st, g, rh, h2, f, x, color,
                (float)omega, k0, rev ? 1 : 0);
        else
            launch_pdl(rbgs_rho_tile_kernel<false, false, V>, gr, dim3(kBX, kVY), 0, st, g, rh, h2, f, x, color,
                (float)omega, k0, rev ? 1 : 0);
        count_launch();
        return;
    }
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

// ---- the product and the restriction over plane tiles, V pairs per lane
//
// The layout of the colour pass over tiles (rbgs_rho_tile_kernel): a block
// applies A to an 8-row tile of one plane (the restriction: of the two planes
// of one coarse plane), every value a V-wide vector load of a half-row, the
// planes above and below read again (from L2) by each plane's tiles.

namespace {

// (A x)/scale of the 2V cells 2t0 .. 2t0+2V-1 of row j, plane k, in cell
// order; C0: colour of cell 2t0 ((j + k) & 1).  Faces in the order x-, x+,
// y-, y+, z-, z+ of op_apply.  X, F: x (and f) of the cells in cell order.
// XP: x is formed on the fly as z + beta x (the flexible CG's direction
// update d = z + beta d fused into the product that reads it; same FMA as
// the separate update, so the same values).
template <bool WITH_F, int V, int C0, bool XP = false, typename RT = float>
__device__ __forceinline__ void tile_apply(const Geo& g, const RT* __restrict__ rh, const float* __restrict__ x,
                                           const float* __restrict__ f, int j, int k, int t0, int lane,
                                           float (&a)[2 * V], float (&X)[2 * V], float (&F)[2 * V],
                                           const float* __restrict__ z = nullptr, float beta = 0.f) {
    const int nx = g.nx, hx = nx / 2, pl = nx * g.ny;
    const int rb = k * pl + j * nx;
    const int o = rb + 2 * t0;
    const int ym = j > 0 ? -nx : (g.ny - 1) * nx, yp = j < g.ny - 1 ? nx : -(g.ny - 1) * nx;
    const int zm = k > 0 ? -pl : (g.nz - 1) * pl, zp = k < g.nz - 1 ? pl : -(g.nz - 1) * pl;
    // half-rows h = 0, 1 at entries t0 .. t0+V-1; entry v of half h is cell
    // 2(t0+v) + (h ^ C0) in this row, 2(t0+v) + (h ^ C0 ^ 1) in the rows and
    // planes next to it
    float h0[V], h1[V];
    auto cells = [&](int off, int c0, float (&out)[2 * V]) {
        ldgv<V>(h0, x + rb + off + t0);
        ldgv<V>(h1, x + rb + off + hx + t0);
        if (XP) {
            float g0[V], g1[V];
            ldgv<V>(g0, z + rb + off + t0);
            ldgv<V>(g1, z + rb + off + hx + t0);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                h0[v] = fmaf(beta, h0[v], g0[v]);
                h1[v] = fmaf(beta, h1[v], g1[v]);
            }
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            out[2 * v] = c0 ? h1[v] : h0[v];
            out[2 * v + 1] = c0 ? h0[v] : h1[v];
        }
    };
    float R[2 * V], Rym[2 * V], Ryp[2 * V], Rzm[2 * V], Rzp[2 * V];
    float Xym[2 * V], Xyp[2 * V], Xzm[2 * V], Xzp[2 * V];
    ldgv<2 * V>(R, rh + o);
    ldgv<2 * V>(Rym, rh + o + ym);
    ldgv<2 * V>(Ryp, rh + o + yp);
    ldgv<2 * V>(Rzm, rh + o + zm);
    ldgv<2 * V>(Rzp, rh + o + zp);
    cells(0, C0, X);
    cells(ym, C0 ^ 1, Xym);
    cells(yp, C0 ^ 1, Xyp);
    cells(zm, C0 ^ 1, Xzm);
    cells(zp, C0 ^ 1, Xzp);
    if (WITH_F) {
        ldgv<V>(h0, f + rb + t0);
        ldgv<V>(h1, f + rb + hx + t0);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            F[2 * v] = C0 ? h1[v] : h0[v];
            F[2 * v + 1] = C0 ? h0[v] : h1[v];
        }
    }
    // cells 2t0-1 (colour C0^1) and 2t0+2V (colour C0) outside the lane's
    // entries, wrapped around the row: from the adjacent lanes, or loaded
    const int tl = t0 > 0 ? t0 - 1 : hx - 1, tr = t0 + V < hx ? t0 + V : t0 + V - hx;
    float xl_ld = __ldg(x + rb + (C0 ? 0 : hx) + tl), xr_ld = __ldg(x + rb + (C0 ? hx : 0) + tr);
    if (XP) {
        xl_ld = fmaf(beta, xl_ld, __ldg(z + rb + (C0 ? 0 : hx) + tl));
        xr_ld = fmaf(beta, xr_ld, __ldg(z + rb + (C0 ? hx : 0) + tr));
    }
    const float rl_ld = ldr(rh + o + (t0 > 0 ? -1 : nx - 1));
    const float rr_ld = ldr(rh + o + (t0 + V < hx ? 2 * V : 2 * V - nx));
    const float xl_sh = __shfl_up_sync(kAll, X[2 * V - 1], 1), rl_sh = __shfl_up_sync(kAll, R[2 * V - 1], 1);
    const float xr_sh = __shfl_down_sync(kAll, X[0], 1), rr_sh = __shfl_down_sync(kAll, R[0], 1);
    const bool left_lane = lane > 0 && t0 > 0, right_lane = lane < 31 && t0 + V < hx;
    const float xl = left_lane ? xl_sh : xl_ld, rl = left_lane ? rl_sh : rl_ld;
    const float xr = right_lane ? xr_sh : xr_ld, rr = right_lane ? rr_sh : rr_ld;
    const bool ym_wall = g.wy && j == 0, yp_wall = g.wy && j == g.ny - 1;
    const bool zm_wall = g.wz && k == 0, zp_wall = g.wz && k == g.nz - 1;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const float bxi = bface(R[2 * v], R[2 * v + 1]);
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int c = 2 * v + m;
            float bxm, bxp, xm, xp;
            if (m == 0) {
                const bool wall = g.wx && t0 + v == 0;
                const float xo = v > 0 ? X[c - 1] : xl, ro = v > 0 ? R[c - 1] : rl;
                bxm = wall ? 0.f : bface(R[c], ro);
                xm = xo;
                bxp = bxi;
                xp = X[c + 1];
            } else {
                const bool wall = g.wx && t0 + v == hx - 1;
                const float xo = v < V - 1 ? X[c + 1] : xr, ro = v < V - 1 ? R[c + 1] : rr;
                bxm = bxi;
                xm = X[c - 1];
                bxp = wall ? 0.f : bface(R[c], ro);
                xp = xo;
            }
            const float bym = ym_wall ? 0.f : bface(R[c], Rym[c]);
            const float byp = yp_wall ? 0.f : bface(R[c], Ryp[c]);
            const float bzm = zm_wall ? 0.f : bface(Rzm[c], R[c]);
            const float bzp = zp_wall ? 0.f : bface(R[c], Rzp[c]);
            const float xc = X[c];
            float s = bxm * (xc - xm);
            s = fmaf(bxp, xc - xp, s);
            s = fmaf(bym, xc - Xym[c], s);
            s = fmaf(byp, xc - Xyp[c], s);
            s = fmaf(bzm, xc - Xzm[c], s);
            s = fmaf(bzp, xc - Xzp[c], s);
            a[c] = s;
        }
    }
}

// The residual restriction's operator sums over the 2 x 2 x 2 children of
// a coarse cell.  Summed over the children, A x keeps only the faces on the
// coarse cell's surface: a face between two children enters once from each
// side with opposite signs.  So each child takes only its faces on that
// surface: along x the pair's outer face (the pairs are the coarse cells'
// x-extents), along y the face away from the other row of the coarse cell
// (row j even: y-, odd: y+), along z likewise (plane k even: z-, odd: z+).
// a: (A x)/scale restricted to those faces for the 2V cells of row j, plane
// k, in cell order; F: f of the same cells.  Three faces a cell instead of
// six, and one y- and one z-neighbour row instead of two.
template <int V, int C0, typename RT>
__device__ __forceinline__ void tile_restrict_faces(const Geo& g, const RT* __restrict__ rh,
                                                    const float* __restrict__ x, const float* __restrict__ f,
                                                    int j, int k, int t0, int lane, float (&a)[2 * V],
                                                    float (&F)[2 * V]) {
    const int nx = g.nx, hx = nx / 2, pl = nx * g.ny;
    const int rb = k * pl + j * nx;
    const int o = rb + 2 * t0;
    const bool jodd = j & 1, kodd = k & 1;
    const int oy = !jodd ? (j > 0 ? -nx : (g.ny - 1) * nx) : (j < g.ny - 1 ? nx : -(g.ny - 1) * nx);
    const int oz = !kodd ? (k > 0 ? -pl : (g.nz - 1) * pl) : (k < g.nz - 1 ? pl : -(g.nz - 1) * pl);
    const bool ywall = g.wy && (!jodd ? j == 0 : j == g.ny - 1);
    const bool zwall = g.wz && (!kodd ? k == 0 : k == g.nz - 1);
    float h0[V], h1[V];
    auto cells = [&](int off, int c0, float (&out)[2 * V]) {
        ldgv<V>(h0, x + rb + off + t0);
        ldgv<V>(h1, x + rb + off + hx + t0);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            out[2 * v] = c0 ? h1[v] : h0[v];
            out[2 * v + 1] = c0 ? h0[v] : h1[v];
        }
    };
    float R[2 * V], Ry[2 * V], Rz[2 * V], X[2 * V], Xy[2 * V], Xz[2 * V];
    ldgv<2 * V>(R, rh + o);
    ldgv<2 * V>(Ry, rh + o + oy);
    ldgv<2 * V>(Rz, rh + o + oz);
    cells(0, C0, X);
    cells(oy, C0 ^ 1, Xy);
    cells(oz, C0 ^ 1, Xz);
    ldgv<V>(h0, f + rb + t0);
    ldgv<V>(h1, f + rb + hx + t0);
#pragma unroll
    for (int v = 0; v < V; ++v) {
        F[2 * v] = C0 ? h1[v] : h0[v];
        F[2 * v + 1] = C0 ? h0[v] : h1[v];
    }
    // cells 2t0-1 and 2t0+2V outside the lane's entries, wrapped around the
    // row: from the adjacent lanes, or loaded
    const int tl = t0 > 0 ? t0 - 1 : hx - 1, tr = t0 + V < hx ? t0 + V : t0 + V - hx;
    const float xl_ld = __ldg(x + rb + (C0 ? 0 : hx) + tl), xr_ld = __ldg(x + rb + (C0 ? hx : 0) + tr);
    const float rl_ld = ldr(rh + o + (t0 > 0 ? -1 : nx - 1));
    const float rr_ld = ldr(rh + o + (t0 + V < hx ? 2 * V : 2 * V - nx));
    const float xl_sh = __shfl_up_sync(kAll, X[2 * V - 1], 1), rl_sh = __shfl_up_sync(kAll, R[2 * V - 1], 1);
    const float xr_sh = __shfl_down_sync(kAll, X[0], 1), rr_sh = __shfl_down_sync(kAll, R[0], 1);
    const bool left_lane = lane > 0 && t0 > 0, right_lane = lane < 31 && t0 + V < hx;
    const float xl = left_lane ? xl_sh : xl_ld, rl = left_lane ? rl_sh : rl_ld;
    const float xr = right_lane ? xr_sh : xr_ld, rr = right_lane ? rr_sh : rr_ld;
#pragma unroll
    for (int v = 0; v < V; ++v) {
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int c = 2 * v + m;
            float xo, ro;
            bool xwall;
            if (m == 0) {
                xwall = g.wx && t0 + v == 0;
                xo = v > 0 ? X[c - 1] : xl;
                ro = v > 0 ? R[c - 1] : rl;
            } else {
                xwall = g.wx && t0 + v == hx - 1;
                xo = v < V - 1 ? X[c + 1] : xr;
                ro = v < V - 1 ? R[c + 1] : rr;
            }
            const float bx = xwall ? 0.f : bface(R[c], ro);
            const float by = ywall ? 0.f : bface(R[c], Ry[c]);
            const float bz = zwall ? 0.f : bface(R[c], Rz[c]);
            const float xc = X[c];
            float sum = bx * (xc - xo);
            sum = fmaf(by, xc - Xy[c], sum);
            sum = fmaf(bz, xc - Xz[c], sum);
            a[c] = sum;
        }
    }
}

}  // namespace

// RESTRICT = false: q = A d on the tiles of np consecutive planes and the
// partial sums of d . q (several planes per block keep the blocks, and so
// the ordered hand-overs of their partial sums, few).
// RESTRICT = true: coarse f = mean over the 2x2x2 children of f - A x; a
// block covers the two planes of one coarse plane (np = 2), and the two fine
// rows of a coarse cell are the warps 2m, 2m+1 of the block, added through
// shared memory.
// blocks per SM the register allocation must allow: the product (with the
// fused direction update) at 4 (64 registers, a few spilled) measured 3 %
// faster than at 3; the restriction on the coarse cells' surface faces at 4
// (64 registers: 43 us against 50 at 3)
#ifndef PARIS_OP_MINB
#define PARIS_OP_MINB 4
#endif
#ifndef PARIS_OP_MINB_R
#define PARIS_OP_MINB_R 4
#endif
// rows per block of the plane-tile restriction (even): two rows measured
// 41.7 us a launch against 43.2 with eight
#ifndef PARIS_RESTRICT_VY
#define PARIS_RESTRICT_VY 2
#endif
constexpr int kVYR = PARIS_RESTRICT_VY;
// the restriction's operator on the coarse cells' surface faces only (0: the
// full stencil of every child)
#ifndef PARIS_RESTRICT_SURFACE
#define PARIS_RESTRICT_SURFACE 1
#endif
constexpr bool kRestrictSurface = PARIS_RESTRICT_SURFACE != 0;
// VB: rows per block (the product's block reduction needs kVY; the
// restriction pairs rows 2m, 2m+1, so VB is even)
template <bool RESTRICT, int V, bool XP = false, typename RT = float, int VB = kVY>
__global__ void __launch_bounds__(kBX* VB, RESTRICT ? PARIS_OP_MINB_R * kVY / VB : PARIS_OP_MINB) op_rho_tile_kernel(Geo g, const RT* __restrict__ rh, float ih2,
                                                             const float* __restrict__ x,
                                                             const float* __restrict__ f,
                                                             float* __restrict__ out, Geo cg,
                                                             double* partials, int np, FinSpec fin,
                                                             const float* __restrict__ z = nullptr,
                                                             const Scal* s = nullptr,
                                                             float* __restrict__ xnew = nullptr, int rev = 0,
                                                             float* __restrict__ eacc = nullptr, int emem = 0) {
    static_assert(RESTRICT ? VB % 2 == 0 : VB == kVY, "rows per block");
    __shared__ float sh[VB][kBX * V];
    pdl_wait();
    // rev: the plane groups in descending order (starting where a previous
    // pass ended); a block's work, and its slot of partial sums, follow its
    // plane group, so the result does not depend on the order
    const int zb = rev ? (int)(gridDim.z - 1 - blockIdx.z) : (int)blockIdx.z;
    const float beta = XP ? (float)s->beta : 0.f;  // XP: x = z + beta x, written to xnew
    // XP with eacc: the inner solution's update e += alpha x of the previous
    // iteration (alpha read before this launch's own finalize replaces it;
    // emem = 0: e not yet written, taken as +0)
    const float alpha_p = (XP && eacc) ? (float)s->alpha : 0.f;
    const int ty = threadIdx.y, lane = threadIdx.x;
    const int j = blockIdx.y * VB + ty;
    const bool row_ok = j < g.ny;
    const int jc = row_ok ? j : g.ny - 1;  // idle rows shadow the last row (no stores)
    const int hx = g.nx / 2;
    const int tv = (blockIdx.x * kBX + lane) * V;
    const bool act = row_ok && tv < hx;
    const int t0 = tv < hx ? tv : hx - V;
    float loc = 0.f;
    float acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = 0.f;
    // e += alpha_p x on the tile row of plane k (both colours, in memory order)
    auto eupd = [&](int k) {
        if (XP && eacc && act) {
            const int rb = (k * g.ny + jc) * g.nx;
            float o0[V], o1[V], e0[V], e1[V];
            ldgv<V>(o0, x + rb + t0);
            ldgv<V>(o1, x + rb + hx + t0);
            if (emem) {
                ldgv<V>(e0, eacc + rb + t0);
                ldgv<V>(e1, eacc + rb + hx + t0);
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) e0[v] = e1[v] = 0.f;
            }
#pragma unroll
            for (int v = 0; v < V; ++v) {
                e0[v] = fmaf(alpha_p, o0[v], e0[v]);
                e1[v] = fmaf(alpha_p, o1[v], e1[v]);
            }
            stv<V>(eacc + rb + t0, e0);
            stv<V>(eacc + rb + hx + t0, e1);
        }
    };
    // plane k's results: q (and the new x) stored, d . q, or the restriction sums
    auto post = [&](int k, const float (&a)[2 * V], const float (&X)[2 * V], const float (&F)[2 * V]) {
        if (!RESTRICT) {
            const int c0 = (jc + k) & 1;
            float Q[2 * V], q0[V], q1[V];
#pragma unroll
            for (int c = 0; c < 2 * V; ++c) Q[c] = ih2 * a[c];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                q0[v] = c0 ? Q[2 * v + 1] : Q[2 * v];
                q1[v] = c0 ? Q[2 * v] : Q[2 * v + 1];
            }
            if (act) {
                const int rb = (k * g.ny + jc) * g.nx;
                stv<V>(out + rb + t0, q0);
                stv<V>(out + rb + hx + t0, q1);
                if (XP) {
                    float d0[V], d1[V];
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        d0[v] = c0 ? X[2 * v + 1] : X[2 * v];
                        d1[v] = c0 ? X[2 * v] : X[2 * v + 1];
                    }
                    stv<V>(xnew + rb + t0, d0);
                    stv<V>(xnew + rb + hx + t0, d1);
                }
#pragma unroll
                for (int c = 0; c < 2 * V; ++c) loc = fmaf(X[c], Q[c], loc);
            }
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] += (F[2 * v] - ih2 * a[2 * v]) + (F[2 * v + 1] - ih2 * a[2 * v + 1]);
        }
    };
    for (int p = 0; p < np; ++p) {
        const int k = zb * np + p;
        if (k >= g.nz) break;  // uniform per block
        eupd(k);
        float a[2 * V], X[2 * V], F[2 * V];
        if constexpr (RESTRICT && kRestrictSurface) {
            if (((jc + k) & 1) == 0)
                tile_restrict_faces<V, 0, RT>(g, rh, x, f, jc, k, t0, lane, a, F);
            else
                tile_restrict_faces<V, 1, RT>(g, rh, x, f, jc, k, t0, lane, a, F);
        } else {
            if (((jc + k) & 1) == 0)
                tile_apply<RESTRICT, V, 0, XP, RT>(g, rh, x, f, jc, k, t0, lane, a, X, F, z, beta);
            else
                tile_apply<RESTRICT, V, 1, XP, RT>(g, rh, x, f, jc, k, t0, lane, a, X, F, z, beta);
        }
        post(k, a, X, F);
    }
    if (RESTRICT) {
#pragma unroll
        for (int v = 0; v < V; ++v) sh[ty][lane * V + v] = acc[v];
        __syncthreads();
        if ((ty & 1) == 0 && act) {
            float cf[V];
#pragma unroll
            for (int v = 0; v < V; ++v) cf[v] = (sh[ty][lane * V + v] + sh[ty + 1][lane * V + v]) * 0.125f;
            stv<V>(out + (zb * cg.ny + (j >> 1)) * cg.nx + t0, cf);
        }
    } else {
        double red[1] = {(double)loc};
        const int op[1] = {0};
        const int64_t blk = ((int64_t)zb * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        block_reduce_store<1>(red, op, partials, blk, ty * kBX + lane);
        finalize_last_block(partials, (int64_t)gridDim.x * gridDim.y * gridDim.z, fin, ty * kBX + lane);
    }
}

#ifndef PARIS_OP_PLANES
#define PARIS_OP_PLANES 16
#endif
// planes per block of the tile product: 16 measured 98 us a launch against 102
// with 8 and 121 with 2
constexpr int kTileOpPlanes = PARIS_OP_PLANES;

int64_t rho0_matvec_blocks(const Geo& g) {
    // the most blocks any segment length (>= 2 planes) gives, or the plane tiles
    const int64_t ring = (int64_t)pair_blocks_x(g) * ((g.ny + kVY - 1) / kVY) * ((g.nz + 1) / 2);
    const int64_t tiles = (int64_t)((g.nx / 2 + 2 * kBX - 1) / (2 * kBX)) * ((g.ny + kVY - 1) / kVY) *
                          ((g.nz + kTileOpPlanes - 1) / kTileOpPlanes);
    return ring > tiles ? ring : tiles;
}

bool rho0_product_fuses(const Geo& g, bool tiles) { return tiles && kTileOpV > 0 && (g.nx / 2) % kTileOpV == 0; }

int64_t launch_matvec_rho_xpby(const Geo& g, const float* rh, double h, const float* z, const float* d, float* dnew,
                               float* q, const Scal* s, double* partials, cudaStream_t st, FinSpec fin, bool rev,
                               float* e, bool emem) {
    constexpr int V = kTileOpV > 0 ? kTileOpV : 2;
    const int hx = g.nx / 2;
    dim3 gr((hx / V + kBX - 1) / kBX, (g.ny + kVY - 1) / kVY, (g.nz + kTileOpPlanes - 1) / kTileOpPlanes);
    launch_pdl(op_rho_tile_kernel<false, V, true>, gr, dim3(kBX, kVY), 0, st, g, rh, (float)(1.0 / (h * h)), d,
               (const float*)nullptr, q, g, partials, kTileOpPlanes, fin, z, s, dnew, rev ? 1 : 0, e, emem ? 1 : 0);
    count_launch();
    return (int64_t)gr.x * gr.y * gr.z;
}

int64_t launch_matvec_rho(const Geo& g, const float* rh, double h, const float* d, float* q,
                          double* partials, cudaStream_t st, FinSpec fin, bool tiles, bool rev) {
    const int hx = g.nx / 2;
    if (tiles && kTileOpV > 0 && hx % kTileOpV == 0) {
        constexpr int V = kTileOpV > 0 ? kTileOpV : 2;
        dim3 gr((hx / V + kBX - 1) / kBX, (g.ny + kVY - 1) / kVY, (g.nz + kTileOpPlanes - 1) / kTileOpPlanes);
        launch_pdl(op_rho_tile_kernel<false, V>, gr, dim3(kBX, kVY), 0, st, g, rh, (float)(1.0 / (h * h)), d,
            (const float*)nullptr, q, g, partials, kTileOpPlanes, fin, (const float*)nullptr, (const Scal*)nullptr,
            (float*)nullptr, rev ? 1 : 0, (float*)nullptr, 0);
        count_launch();
        return (int64_t)gr.x * gr.y * gr.z;
    }
    const int seg = segment_planes(g, g.nz, (const void*)op_rho_kernel<false>);
    dim3 gr(pair_blocks_x(g), (g.ny + kVY - 1) / kVY, (g.nz + seg - 1) / seg);
    op_rho_kernel<false><<<gr, dim3(kBX, kVY), 0, st>>>(g, rh, (float)(1.0 / (h * h)), d, nullptr, q, g,
                                                        partials, seg, fin);
    count_launch();
    return (int64_t)gr.x * gr.y * gr.z;
}

void launch_restrict_rho(const Geo& g, const float* rh, double h, const float* f, const float* x,
                         const Geo& cg, float* fc, cudaStream_t st, bool tiles, const __half* rh16, bool rev) {
    const int hx = g.nx / 2;
    if (tiles && kTileOpV > 0 && hx % kTileOpV == 0) {
        constexpr int V = kTileOpV > 0 ? kTileOpV : 2;
        dim3 gr((hx / V + kBX - 1) / kBX, (g.ny + kVYR - 1) / kVYR, g.nz / 2);
        if (rh16)  // the V-cycle's restriction from FP16 rho/2
            launch_pdl(op_rho_tile_kernel<true, V, false, __half, kVYR>, gr, dim3(kBX, kVYR), 0, st, g, rh16,
                       (float)(1.0 / (h * h)), x, f, fc, cg, (double*)nullptr, 2, no_fin(), (const float*)nullptr,
                       (const Scal*)nullptr, (float*)nullptr, rev ? 1 : 0, (float*)nullptr, 0);
        else
            launch_pdl(op_rho_tile_kernel<true, V, false, float, kVYR>, gr, dim3(kBX, kVYR), 0, st, g, rh,
                (float)(1.0 / (h * h)), x, f,
                fc, cg, (double*)nullptr, 2, no_fin(), (const float*)nullptr, (const Scal*)nullptr, (float*)nullptr,
                rev ? 1 : 0, (float*)nullptr, 0);
        count_launch();
        return;
    }
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
__global__ void prolong_split_kernel(Geo fg, Geo cg, const float* __restrict__ xc, float* __restrict__ x, int rev) {
    pdl_wait();
    const int hx = fg.nx / 2;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = rev ? (int)(gridDim.z - 1 - blockIdx.z) : (int)blockIdx.z;  // rev: descending planes
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

void launch_prolong_split(const Geo& fine, const Geo& coarse, const float* xc, float* x, cudaStream_t st, bool rev) {
    const int hx = fine.nx / 2;
    const bool v4 = hx % 4 == 0 && ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(xc)) & 15) == 0;
    const int per = v4 ? 4 : 1;
    dim3 blk(32, 8);
    dim3 gr((hx / per + 31) / 32, (fine.ny + 7) / 8, fine.nz);
    if (v4) launch_pdl(prolong_split_kernel<4>, gr, blk, 0, st, fine, coarse, xc, x, rev ? 1 : 0);
    else launch_pdl(prolong_split_kernel<1>, gr, blk, 0, st, fine, coarse, xc, x, rev ? 1 : 0);
    count_launch();
}

// --------------------------------------------------- level-1 coefficients ---

// beta of the level with every axis halved: the mean of the four fine faces
// that tile each coarse face, times (h0/h1)^2 = 1/4 and the fine scale
// 1/h0^2 (the coarse arrays hold scaled coefficients).
template <int AXIS>
__global__ void coarse_beta_rho_kernel(Geo fg, const float* __restrict__ rh, float scale, Geo cg,
                                       float* __restrict__ out, __half* __restrict__ out16, float s16) {
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
            if (out16) out16[t] = __float2half_rn(0.f);
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
        if (out16) out16[t] = __float2half_rn(s * s16);  // the sum times a power of two
    }
}

void launch_coarse_beta_rho(const Geo& fine, const float* rh, double h, const Geo& coarse, float* out[3],
                            cudaStream_t st, __half* const out16[3], float s16) {
    // mean of 4 faces (1/4) x (h0/h1)^2 (1/4) x 1/h0^2
    const float scale = (float)(1.0 / (16.0 * h * h));
    for (int a = 0; a < 3; ++a) {
        const unsigned nb = (unsigned)elementwise_blocks(coarse.nface(a));
        __half* o16 = out16 ? out16[a] : nullptr;
        if (a == 0) coarse_beta_rho_kernel<0><<<nb, kRedThreads, 0, st>>>(fine, rh, scale, coarse, out[0], o16, s16);
        if (a == 1) coarse_beta_rho_kernel<1><<<nb, kRedThreads, 0, st>>>(fine, rh, scale, coarse, out[1], o16, s16);
        if (a == 2) coarse_beta_rho_kernel<2><<<nb, kRedThreads, 0, st>>>(fine, rh, scale, coarse, out[2], o16, s16);
    }
    count_launch(3);
}

}  // namespace paris
