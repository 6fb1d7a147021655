// The FP64 refinement step of the mixed form in double-float arithmetic.
//
// After an FP32 inner solve of A e = r32 (r32 = 2^a r, a an integer), the
// correction is d = 2^-a e and the refinement step is
//   x <- x + d,   r <- r - A d,
// the residual updated rather than recomputed as f - A x.  A d is needed to
// about 1e-11 relative (|A d| is about |r|, and r must stay accurate to
// ~1e-16 |f|); this kernel evaluates it in pairs of FP32 numbers ("double-
// float", about 48 significant bits) on the FP32 pipe, which on this GPU is
// 64 times faster than the FP64 one, from the half-densities rho/2 held as
// hi + lo FP32 pairs (written by the face-coefficient kernel from the FP64
// values).  The error-free transformations are Knuth's two-sum and the
// FMA-based two-product; 1/(rh_L + rh_R) is one FP32 reciprocal refined to
// second order; intermediate pairs are left unnormalised where the next step
// reads both halves, and the six face terms are summed with one two-sum
// chain plus one error accumulator.  Only the updates of x and r use FP64
// instructions (3 per cell, against 14 for a full FP64 residual).  The same pass writes the next inner right-hand side
// r32 = 2^b r with 2^b from max |r| before the step, and the norms of r.
#include "kernels.cuh"

namespace paris {

namespace {

constexpr int kTX = 32, kTY = 8, kZ = 16;  // 16 cells per thread along z

struct F2 {
    float hi, lo;
};

// a + b = s + err exactly (Knuth)
__device__ __forceinline__ F2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
    return F2{s, err};
}

// 2^sh (hi + lo) in FP64: exact widenings with the exponent shift (integer
// operations), one FP64 add
__device__ __forceinline__ double pair_to_double_scaled(float hi, float lo, int sh) {
    return f2d_scaled(hi, sh) + f2d_scaled(lo, sh);
}

// e with v = m 2^e, m in [0.5, 1), for a positive normal v (from the IEEE
// exponent field); 0 otherwise
__device__ __forceinline__ int exponent_of(double v) {
    const int b = (__double2hiint(v) >> 20) & 0x7ff;
    return (b == 0 || b == 0x7ff) ? 0 : b - 1022;
}

// One face term beta_f (e_c - e_nb) added to the sum S + E: rho/2 of the cell
// (rc) and of the neighbour (rq) as (hi, lo) pairs
__device__ __forceinline__ void face_term(float2 rc, float2 rq, float ec, float eq, float& S, float& E) {
    // rho_L/2 + rho_R/2 as an unnormalised pair
    const F2 sum = two_sum(rc.x, rq.x);
    const float slo = __fadd_rn(sum.lo, __fadd_rn(rc.y, rq.y));
    // beta = 1/sum: y0 to ~1 ulp, t = 1 - sum y0, beta = y0 + y0 (t + t^2)
    float y0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(sum.hi));
    float t = __fmaf_rn(-sum.hi, y0, 1.0f);
    t = __fmaf_rn(-slo, y0, t);
    const float blo = __fmul_rn(y0, __fmaf_rn(t, t, t));
    // e_c - e_nb exactly, then the product with beta
    const F2 d = two_sum(ec, -eq);
    const float ph = __fmul_rn(y0, d.hi);
    float plo = __fmaf_rn(y0, d.hi, -ph);
    plo = __fmaf_rn(y0, d.lo, __fmaf_rn(blo, d.hi, plo));
    const F2 a = two_sum(S, ph);
    S = a.hi;
    E = __fadd_rn(E, __fadd_rn(a.lo, plo));
}

}  // namespace

// One refinement step on the finest level (see the file comment).  r_old and
// r_new may be the same array (each cell reads and writes only its own r).
// rh2 holds rho/2 per cell as (hi, lo) FP32 pairs.  The squared norm of r is
// accumulated from the O(1)-scaled r32 in FP32 and unscaled in the finalize.
__global__ void __launch_bounds__(kTX* kTY) refine_rho_kernel(Geo g, const float2* __restrict__ rh2,
                                                            float ih2_hi, float ih2_lo,
                                                            const float* __restrict__ e,
                                                            const double* r_old, double* r_new,
                                                            double* __restrict__ x, float* __restrict__ r32,
                                                            const Scal* s, double* partials, FinSpec fin, int rev,
                                                            int emem, const float* __restrict__ dpend) {
    pdl_wait();
    const int zb = rev ? (int)(gridDim.z - 1 - blockIdx.z) : (int)blockIdx.z;  // rev: descending plane chunks
    const int i = blockIdx.x * kTX + threadIdx.x;
    const int j = blockIdx.y * kTY + threadIdx.y;
    float l2 = 0.f;
    unsigned long long rmax_k = 0;
    unsigned nf = 0;
    if (i < g.nx && j < g.ny) {
        const int sa = (int)s->scale_exp;  // r32 of this inner solve = 2^sa r
        // the inner solution at entry p: e (0 when not yet written), plus the
        // pending last update alpha dpend (the same FMA the inner loop's update
        // would have made)
        const float ap = dpend ? (float)s->alpha : 0.f;
        auto ev = [&](int p) {
            const float v = emem ? __ldg(e + p) : 0.f;
            return dpend ? __fmaf_rn(ap, __ldg(dpend + p), v) : v;
        };
        const int sb = -exponent_of(s->rinf);  // next r32 = 2^sb r (the scale of FIN_SCALE)
        const int nx = g.nx, ny = g.ny, nz = g.nz, pl = nx * ny;
        // neighbour offsets along x and y (periodic wrap; a wall side points at
        // the cell itself and its face is skipped)
        const bool xlo = i == 0, xhi = i == nx - 1, ylo = j == 0, yhi = j == ny - 1;
        const int oxm = !xlo ? -1 : (g.wx ? 0 : nx - 1), oxp = !xhi ? 1 : (g.wx ? 0 : -(nx - 1));
        const int oym = !ylo ? -nx : (g.wy ? 0 : (ny - 1) * nx), oyp = !yhi ? nx : (g.wy ? 0 : -(ny - 1) * nx);
        const bool wxm = g.wx && xlo, wxp = g.wx && xhi, wym = g.wy && ylo, wyp = g.wy && yhi;
        // e and r32 are colour-split: cell i of a row at i/2, plus nx/2 for
        // colour (i+j+k) odd.  The x-neighbours' entries within the row (the
        // other colour, so the half is fixed per plane below)
        const int hx = nx / 2;
        const int tx = i >> 1;
        const int txm = (xlo ? nx - 1 : i - 1) >> 1, txp = (xhi ? 0 : i + 1) >> 1;
        const int k0 = zb * kZ, k1 = min(k0 + kZ, nz);
        for (int k = k0; k < k1; ++k) {
            const int c = (k * ny + j) * nx + i;
            const bool zlo = k == 0, zhi = k == nz - 1;
            const int ozm = !zlo ? -pl : (g.wz ? 0 : (nz - 1) * pl), ozp = !zhi ? pl : (g.wz ? 0 : -(nz - 1) * pl);
            const bool wzm = g.wz && zlo, wzp = g.wz && zhi;
            const int odd = (i + j + k) & 1;
            const int rb = c - i;
            const int sc = rb + (odd ? hx : 0) + tx;           // this cell
            const int so = rb + (odd ? 0 : hx);                // other colour's half of this row
            const int sn = so + tx;                            // y and z neighbours: same entry, other half
            const float2 rc = __ldg(rh2 + c);
            const float ec = ev(sc);
            // sum over the faces of beta_f (e_c - e_nb) as S + E: S the running
            // FP32 sum of the leading products (two-sum), E every rounding
            // error and low part (faces x-, x+, y-, y+, z-, z+)
            float S = 0.f, E = 0.f;
            if (!wxm) face_term(rc, __ldg(rh2 + c + oxm), ec, ev(so + txm), S, E);
            if (!wxp) face_term(rc, __ldg(rh2 + c + oxp), ec, ev(so + txp), S, E);
            if (!wym) face_term(rc, __ldg(rh2 + c + oym), ec, ev(sn + oym), S, E);
            if (!wyp) face_term(rc, __ldg(rh2 + c + oyp), ec, ev(sn + oyp), S, E);
            if (!wzm) face_term(rc, __ldg(rh2 + c + ozm), ec, ev(sn + ozm), S, E);
            if (!wzp) face_term(rc, __ldg(rh2 + c + ozp), ec, ev(sn + ozp), S, E);
            // A d = 2^-sa (S + E) ih2, the product as a pair, the power of two
            // applied exactly on the FP64 side
            const float qh = __fmul_rn(S, ih2_hi);
            float ql = __fmaf_rn(S, ih2_hi, -qh);
            ql = __fmaf_rn(S, ih2_lo, __fmaf_rn(E, ih2_hi, ql));
            const double ad = pair_to_double_scaled(qh, ql, -sa);
            const double rn = r_old[c] - ad;
            r_new[c] = rn;
            x[c] += f2d_scaled(ec, -sa);
            const float rs = d2f_scaled(rn, sb);
            r32[sc] = rs;
            l2 = __fmaf_rn(rs, rs, l2);
            const unsigned long long kr = abs_key(rn);
            rmax_k = kr > rmax_k ? kr : rmax_k;
            nf += key_nonfinite(kr);
        }
    }
    const int tid = threadIdx.y * kTX + threadIdx.x;
    const int64_t blk = ((int64_t)zb * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    block_reduce_skc<float>(l2, rmax_k, nf, partials, blk, tid);
    finalize_last_block(partials, (int64_t)gridDim.x * gridDim.y * gridDim.z, fin, tid);
}

void launch_refine_rho(const Geo& g, const float2* rh2, double h, const float* e, const double* r_old,
                       double* r_new, double* x, float* r32, Scal* s, double* partials, cudaStream_t st, bool rev,
                       bool emem, const float* dpend) {
    // 1/h^2 as an FP32 pair
    const double ih2d = 1.0 / (h * h);
    const float hi = (float)ih2d;
    const float lo = (float)(ih2d - (double)hi);
    dim3 gr((g.nx + kTX - 1) / kTX, (g.ny + kTY - 1) / kTY, (g.nz + kZ - 1) / kZ);
    launch_pdl(refine_rho_kernel, gr, dim3(kTX, kTY), 0, st, g, rh2, hi, lo, e, r_old, r_new, x, r32, s,
        partials, FinSpec{s, 3, 2, FIN_REFINE, 0.0}, rev ? 1 : 0, emem ? 1 : 0, dpend);
    count_launch();
}

}  // namespace paris
