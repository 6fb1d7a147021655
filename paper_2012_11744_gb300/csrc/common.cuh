// Shared device-side definitions of the projection library: grid geometry,
// face indexing, the 7-point variable-coefficient stencil and deterministic
// block reductions.  Internal header (not part of the C ABI).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace paris {

constexpr int kRedThreads = 256;  // threads of every reducing kernel's block

// One grid level: cells per axis and wall flags.  Cell (i,j,k) lives at
// (k*ny + j)*nx + i; face arrays extend the face axis by one when that axis
// has walls (entries 0 and n are the wall faces).
struct Geo {
    int nx, ny, nz;
    int wx, wy, wz;

    __host__ __device__ int64_t ncell() const { return (int64_t)nx * ny * nz; }
    __host__ __device__ int64_t nface(int axis) const {
        return (int64_t)(nx + (axis == 0 ? wx : 0)) * (ny + (axis == 1 ? wy : 0)) *
               (nz + (axis == 2 ? wz : 0));
    }
    __host__ __device__ int64_t cidx(int i, int j, int k) const {
        return ((int64_t)k * ny + j) * nx + i;
    }
    __host__ __device__ int64_t fx(int i, int j, int k) const {
        return ((int64_t)k * ny + j) * (nx + wx) + i;
    }
    __host__ __device__ int64_t fy(int i, int j, int k) const {
        return ((int64_t)k * (ny + wy) + j) * nx + i;
    }
    __host__ __device__ int64_t fz(int i, int j, int k) const {
        return ((int64_t)k * ny + j) * nx + i;
    }
};

// Coefficient set of one level: face arrays and a uniform scale (1/h^2 for
// arrays holding beta itself, 1 for arrays that are already scaled), and an
// optional per-cell diagonal excess sig in the units of the face arrays: the
// operator is  (A x)_c = scale (sum_f beta_f (x_c - x_nb) + sig_c x_c),  the
// form a Dirichlet condition at a cut face takes (Sec. 3.7.5); null: none.
template <typename T>
struct Coef {
    const T* bx;
    const T* by;
    const T* bz;
    T scale;
    const T* sig = nullptr;
};

// Neighbour indices and + face index along one axis of length n.  Along a
// wall axis the missing neighbour is clamped onto the cell itself; its face
// coefficient is forced to zero (Neumann by coefficient zeroing).
struct AxisNb {
    int m, p, fp;   // minus neighbour, plus neighbour, index of the + face
    bool wm, wp;    // minus / plus face is a wall
};

__host__ __device__ inline AxisNb axis_nb(int i, int n, int wall) {
    AxisNb a;
    a.wm = wall && i == 0;
    a.wp = wall && i == n - 1;
    a.m = i > 0 ? i - 1 : (wall ? 0 : n - 1);
    a.p = i + 1 < n ? i + 1 : (wall ? n - 1 : 0);
    a.fp = (i + 1 < n || wall) ? i + 1 : 0;
    return a;
}

// The six face coefficients (unscaled) around cell (i,j,k) and the neighbour
// cell indices, in the order x-, x+, y-, y+, z-, z+.
template <typename T>
struct Stencil {
    T b[6];
    int64_t nb[6];
};

template <typename T>
__device__ inline void load_stencil(const Geo& g, const Coef<T>& cf, int i, int j, int k,
                                    Stencil<T>& s) {
    AxisNb ax = axis_nb(i, g.nx, g.wx);
    AxisNb ay = axis_nb(j, g.ny, g.wy);
    AxisNb az = axis_nb(k, g.nz, g.wz);
    s.b[0] = ax.wm ? T(0) : cf.bx[g.fx(i, j, k)];
    s.b[1] = ax.wp ? T(0) : cf.bx[g.fx(ax.fp, j, k)];
    s.b[2] = ay.wm ? T(0) : cf.by[g.fy(i, j, k)];
    s.b[3] = ay.wp ? T(0) : cf.by[g.fy(i, ay.fp, k)];
    s.b[4] = az.wm ? T(0) : cf.bz[g.fz(i, j, k)];
    s.b[5] = az.wp ? T(0) : cf.bz[g.fz(i, j, az.fp)];
    s.nb[0] = g.cidx(ax.m, j, k);
    s.nb[1] = g.cidx(ax.p, j, k);
    s.nb[2] = g.cidx(i, ay.m, k);
    s.nb[3] = g.cidx(i, ay.p, k);
    s.nb[4] = g.cidx(i, j, az.m);
    s.nb[5] = g.cidx(i, j, az.p);
}

// Coefficient loads from FP16, FP32 or FP64 storage.
__device__ inline float ldc(const __half* p) { return __half2float(*p); }
__device__ inline float ldc(const float* p) { return *p; }
__device__ inline double ldc(const double* p) { return *p; }

// load_stencil for coefficient arrays stored in another type TB (converted to T)
template <typename T, typename TB>
__device__ inline void load_stencil_as(const Geo& g, const TB* bx, const TB* by, const TB* bz,
                                       int i, int j, int k, Stencil<T>& s) {
    AxisNb ax = axis_nb(i, g.nx, g.wx);
    AxisNb ay = axis_nb(j, g.ny, g.wy);
    AxisNb az = axis_nb(k, g.nz, g.wz);
    s.b[0] = ax.wm ? T(0) : (T)ldc(bx + g.fx(i, j, k));
    s.b[1] = ax.wp ? T(0) : (T)ldc(bx + g.fx(ax.fp, j, k));
    s.b[2] = ay.wm ? T(0) : (T)ldc(by + g.fy(i, j, k));
    s.b[3] = ay.wp ? T(0) : (T)ldc(by + g.fy(i, ay.fp, k));
    s.b[4] = az.wm ? T(0) : (T)ldc(bz + g.fz(i, j, k));
    s.b[5] = az.wp ? T(0) : (T)ldc(bz + g.fz(i, j, az.fp));
    s.nb[0] = g.cidx(ax.m, j, k);
    s.nb[1] = g.cidx(ax.p, j, k);
    s.nb[2] = g.cidx(i, ay.m, k);
    s.nb[3] = g.cidx(i, ay.p, k);
    s.nb[4] = g.cidx(i, j, az.m);
    s.nb[5] = g.cidx(i, j, az.p);
}

// Same result as load_stencil_as with 32-bit index arithmetic (valid while
// every face array of the level holds fewer than 2^31 entries): the cell and
// face offsets of the six neighbours follow from the cell offset by
// additions, with wrap-around or clamping at the domain edges.
template <typename T, typename TB>
__device__ inline void load_stencil_fast(const Geo& g, const TB* bx, const TB* by, const TB* bz,
                                         int i, int j, int k, Stencil<T>& s, int& cell) {
    const int nx = g.nx, ny = g.ny, nz = g.nz, pl = nx * ny;
    const int row = k * ny + j;
    const int c = row * nx + i;
    cell = c;
    const bool xlo = i == 0, xhi = i == nx - 1;
    const int fx = row * (nx + g.wx) + i;
    s.b[0] = (g.wx && xlo) ? T(0) : (T)ldc(bx + fx);
    s.b[1] = (g.wx && xhi) ? T(0) : (T)ldc(bx + ((!xhi || g.wx) ? fx + 1 : fx - (nx - 1)));
    s.nb[0] = !xlo ? c - 1 : (g.wx ? c : c + (nx - 1));
    s.nb[1] = !xhi ? c + 1 : (g.wx ? c : c - (nx - 1));
    const bool ylo = j == 0, yhi = j == ny - 1;
    const int fy = (k * (ny + g.wy) + j) * nx + i;
    s.b[2] = (g.wy && ylo) ? T(0) : (T)ldc(by + fy);
    s.b[3] = (g.wy && yhi) ? T(0) : (T)ldc(by + ((!yhi || g.wy) ? fy + nx : fy - (ny - 1) * nx));
    s.nb[2] = !ylo ? c - nx : (g.wy ? c : c + (ny - 1) * nx);
    s.nb[3] = !yhi ? c + nx : (g.wy ? c : c - (ny - 1) * nx);
    const bool zlo = k == 0, zhi = k == nz - 1;
    s.b[4] = (g.wz && zlo) ? T(0) : (T)ldc(bz + c);
    s.b[5] = (g.wz && zhi) ? T(0) : (T)ldc(bz + ((!zhi || g.wz) ? c + pl : c - (nz - 1) * pl));
    s.nb[4] = !zlo ? c - pl : (g.wz ? c : c + (nz - 1) * pl);
    s.nb[5] = !zhi ? c + pl : (g.wz ? c : c - (nz - 1) * pl);
}

// (A x)_c with A = -L: scale * sum_f beta_f (x_c - x_nb)  (difference form,
// which keeps the FP64 residual accurate when x is smooth).
template <typename T>
__device__ inline T apply_A(const Stencil<T>& s, const T* __restrict__ x, T xc, T scale) {
    T acc = s.b[0] * (xc - x[s.nb[0]]);
#pragma unroll
    for (int q = 1; q < 6; ++q) acc = fma(s.b[q], xc - x[s.nb[q]], acc);
    return scale * acc;
}

// The faces of apply_A selected by mask (bit q: face q), in the same order.
// Summed over the children of a coarse cell, A x keeps only the faces on the
// coarse cell's surface (a face between two children enters once from each
// side with opposite signs): the restrictions take those faces only.
template <typename T>
__device__ inline T apply_A_faces(const Stencil<T>& s, const T* __restrict__ x, T xc, T scale, unsigned mask) {
    T acc = T(0);
#pragma unroll
    for (int q = 0; q < 6; ++q)
        if ((mask >> q) & 1u) acc = fma(s.b[q], xc - x[s.nb[q]], acc);
    return scale * acc;
}

// the faces of child (di, dj, dk) of a coarse cell with factors (f0, f1, f2)
// on the coarse cell's surface: - face of the first child along an axis, +
// face of the last
__device__ inline unsigned surface_faces(int di, int dj, int dk, int f0, int f1, int f2) {
    return (di == 0 ? 1u : 0u) | (di == f0 - 1 ? 2u : 0u) | (dj == 0 ? 4u : 0u) | (dj == f1 - 1 ? 8u : 0u) |
           (dk == 0 ? 16u : 0u) | (dk == f2 - 1 ? 32u : 0u);
}

// 1 / sum of the six face coefficients (the red-black sweeps' inverse diagonal)
__device__ inline float rcp_rn(float d) { return __frcp_rn(d); }  // == 1.0f / d
__device__ inline double rcp_rn(double d) { return 1.0 / d; }

template <typename T>
__device__ inline T inv_sum6(const T (&b)[6]) {
    const T d = ((b[0] + b[1]) + (b[2] + b[3])) + (b[4] + b[5]);
    return d > T(0) ? rcp_rn(d) : T(0);
}

// |v| as an integer key: for non-negative doubles (infinities and NaNs
// included) the order of the bit patterns is the numeric order, so running
// maxima of magnitudes and the non-finite test need no FP64 instruction (the
// FP64 pipe runs at 1/64 of the FP32 rate on this GPU).
__device__ inline unsigned long long abs_key(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
}
__device__ inline unsigned key_nonfinite(unsigned long long k) { return k >= 0x7ff0000000000000ULL ? 1u : 0u; }
__device__ inline double key_value(unsigned long long k) { return __longlong_as_double((long long)k); }

// Conversions between FP64 and FP32 with a power-of-two scaling, written
// with integer operations on the IEEE-754 fields: the hardware conversions
// run on the FP64 pipe at about a fifth of its FMA rate on this GPU.
//
// float(v * 2^s): round to nearest, ties to even, for results in the FP32
// normal range; smaller results flush to a signed zero, larger ones give a
// signed infinity; infinities stay infinite and NaN stays NaN.
__device__ inline float d2f_scaled(double v, int s) {
    const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu);
    if (e == 0x7ff) return __int_as_float((int)(sign | 0x7f800000u | (((hi & 0xfffffu) | lo) ? 0x400000u : 0u)));
    const int fe = e - 896 + s;  // FP32 biased exponent (FP64 bias 1023, FP32 bias 127)
    if (e == 0 || fe <= 0) return __int_as_float((int)sign);
    if (fe >= 255) return __int_as_float((int)(sign | 0x7f800000u));
    // the 23 leading fraction bits; round on the 29 dropped ones (a carry out
    // of the fraction correctly increments the exponent)
    const unsigned frac = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu;
    unsigned bits = ((unsigned)fe << 23) | frac;
    if (rem > 0x10000000u || (rem == 0x10000000u && (frac & 1u))) bits += 1u;
    return __int_as_float((int)(sign | bits));
}

// (double)v * 2^s, exact for normal v whose scaled value is an FP64 normal
// number; FP32 subnormals flush to a signed zero; infinities and NaN are kept.
__device__ inline double f2d_scaled(float v, int s) {
    const unsigned b = (unsigned)__float_as_int(v);
    const unsigned sign = b & 0x80000000u;
    const int e = (int)((b >> 23) & 0xffu);
    const unsigned frac = b & 0x7fffffu;
    if (e == 0xff) return __hiloint2double((int)(sign | 0x7ff00000u | (frac ? 0x80000u : 0u)), 0);
    const int de = e + 896 + s;  // FP64 biased exponent
    if (e == 0 || de <= 0) return __hiloint2double((int)sign, 0);
    if (de >= 0x7ff) return __hiloint2double((int)(sign | 0x7ff00000u), 0);
    return __hiloint2double((int)(sign | ((unsigned)de << 20) | (frac >> 3)), (int)(frac << 29));
}

// Programmatic dependent launch: a kernel launched with launch_pdl may start
// while the kernel before it on the stream is finishing; it waits here for
// that kernel's completion (and its memory) before touching anything the
// earlier kernel writes.  Without the launch attribute the wait returns at
// once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ------------------------------------------------------------ reductions ---

__device__ inline double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ inline double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Reduce NV values over a block of kRedThreads threads (ops: 0 = sum,
// 1 = max) in a fixed order and store them as this block's partials at
// partials[NV*block + q].  Deterministic: the order depends only on the
// thread layout.
template <int NV>
__device__ inline void block_reduce_store(double (&v)[NV], const int (&op)[NV], double* partials,
                                          int64_t block, int tid) {
    __shared__ double sh[kRedThreads / 32][NV];
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = op[q] ? warp_max(v[q]) : warp_sum(v[q]);
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) sh[wid][q] = v[q];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double t = lane < kRedThreads / 32 ? sh[lane][q] : (op[q] ? 0.0 : 0.0);
            t = op[q] ? warp_max(t) : warp_sum(t);
            if (lane == 0) partials[NV * block + q] = t;
        }
    }
}

// Block reduction of one sum, one magnitude key (max) and one count, stored as
// the three partials (sum, key_value(max), count) of this block.  Keys and
// counts are reduced with integer warp reductions and an FP32 sum with FP32
// shuffles, so only the sum of type S uses that type's pipe; fixed order.
template <typename S>
__device__ inline void block_reduce_skc(S sum, unsigned long long key, unsigned cnt, double* partials,
                                        int64_t block, int tid) {
    __shared__ double sh_s[kRedThreads / 32];
    __shared__ unsigned long long sh_k[kRedThreads / 32];
    __shared__ unsigned sh_c[kRedThreads / 32];
    const unsigned all = 0xffffffffu;
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(all, sum, o);
    const unsigned khi = __reduce_max_sync(all, (unsigned)(key >> 32));
    const unsigned klo = __reduce_max_sync(all, (unsigned)(key >> 32) == khi ? (unsigned)key : 0u);
    cnt = __reduce_add_sync(all, cnt);
    if (lane == 0) {
        sh_s[wid] = (double)sum;
        sh_k[wid] = ((unsigned long long)khi << 32) | klo;
        sh_c[wid] = cnt;
    }
    __syncthreads();
    if (tid == 0) {
        double ts = 0.0;
        unsigned long long tk = 0;
        unsigned tc = 0;
        for (int w = 0; w < kRedThreads / 32; ++w) {
            ts += sh_s[w];
            tk = sh_k[w] > tk ? sh_k[w] : tk;
            tc += sh_c[w];
        }
        partials[3 * block + 0] = ts;
        partials[3 * block + 1] = key_value(tk);
        partials[3 * block + 2] = (double)tc;
    }
}

}  // namespace paris
