// Finest-level colour pass with TMA plane staging.
//
// The red-black colour pass of the mixed projection step (Sec. 3.7.1, the
// update of Eq. eq:beta_pressure over one colour, with over-relaxation) on
// the finest level, whose FP32 operator is rebuilt from rho/2 in registers
// (beta_f = 1/(rh_L + rh_R), Eq. muH).  Same vectors, same colour-split
// layout and the same arithmetic, operation by operation, as the register
// plane-tile kernel in rho0.cu (rbgs_rho_tile_kernel): the two give
// bit-identical x.
//
// What differs is how the bytes arrive.  A CTA of R warps owns a tile of R
// rows of one plane and marches it through z; each plane's rows of rho/2, of
// the other colour's x, of the updated colour's x and of f are copied into a
// ring of S shared-memory slots by bulk asynchronous copies (cp.async.bulk,
// the TMA engine's linear mode: every row is contiguous, so one copy moves a
// row and no tensor map is needed), each slot completing on its own
// mbarrier.  One thread issues a plane's copies; while the CTA updates plane
// k from slots k-1, k, k+1, the copies of the planes after k+1 are in flight.
// The CTA thus keeps several planes' bytes in flight with no registers held
// for them, and reads every plane from DRAM once (the tile's two halo rows
// are shared with the neighbouring tiles and mostly come from L2).
//
// Grid: persistent, (SMs) x (resident CTAs per SM); the (tile, plane) work
// items of the pass are split into equal contiguous chunks, one per CTA, so
// a chunk is a run of planes of one tile or the end of one tile's run and
// the start of the next (the ring restarts at a tile boundary).
//
// Every wait on an mbarrier is bounded in time: a wait that gives up sets
// the context's wait_fail word (read by the host after the pass, reported as
// PARIS_ERR_TIMEOUT), the CTA waits with the same bound for its copies in
// flight and returns without writing x.
#include "kernels.cuh"

namespace paris {

namespace {

#ifndef PARIS_STAGE_ROWS
#define PARIS_STAGE_ROWS 8
#endif
#ifndef PARIS_STAGE_SLOTS
#define PARIS_STAGE_SLOTS 4
#endif
constexpr int kStageRows = PARIS_STAGE_ROWS;    // R: rows per tile, one warp each
constexpr int kStageSlots = PARIS_STAGE_SLOTS;  // S: planes held in the ring (S - 2 in flight)
constexpr long long kWaitCycles = 2000000000LL;  // about one second at 2 GHz

__device__ __forceinline__ float rcp_approx(float v) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v));
    return y;
}
__device__ __forceinline__ float bface(float a, float b) { return rcp_approx(a + b); }

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase of the given parity to complete, at most kWaitCycles.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_test(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}
// One bulk copy global -> shared (16-byte aligned, a multiple of 16 bytes),
// completing `bytes` on the mbarrier.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Shared-memory slot of one plane (floats): rh rows j0-1 .. j0+R (R+2 full
// rows, cell order), then the other colour's half-rows of x of the same rows.
// These are the values a plane's tile reads again as the neighbours of the
// planes above and below; the updated colour's x and f are read once, by
// their own plane, straight into registers.
struct SlotLayout {
    int nx, hx;
    int rh, xo, floats;  // offsets in floats; floats = slot size
};
__host__ __device__ inline SlotLayout slot_layout(int nx, int R) {
    SlotLayout s;
    s.nx = nx;
    s.hx = nx / 2;
    s.rh = 0;
    s.xo = s.rh + (R + 2) * nx;
    s.floats = s.xo + (R + 2) * s.hx;
    return s;
}

struct StageArgs {
    Geo g;
    const float* rh;
    const float* f;
    float* x;
    float h2, omega;
    int col;     // the colour updated
    int k0, k1;  // planes of the pass
    int zchunks; // CTAs along z per tile
    unsigned* fail;
};

// Issue the copies of plane kk (wrapped) of tile j0 into a slot: thread 0
// posts the byte count, then the lanes of warp 0 issue one row each.
template <int R, bool ZERO>
__device__ __forceinline__ void issue_plane(const StageArgs& a, const SlotLayout& L, float* slot, uint32_t bar,
                                            int j0, int kk) {
    const int nx = a.g.nx, hx = nx / 2, ny = a.g.ny, nz = a.g.nz;
    kk = kk < 0 ? kk + nz : (kk >= nz ? kk - nz : kk);
    const int lane = threadIdx.x & 31;
    constexpr int nrh = R + 2, nxo = ZERO ? 0 : R + 2;
    constexpr int ncopy = nrh + nxo;
    if (threadIdx.x == 0) mbar_arrive_expect(bar, 4u * (uint32_t)(nrh * nx + nxo * hx));
    __syncwarp();
    const int ocol = a.col ? 0 : hx;  // the other colour's half-row
    for (int c = lane; c < ncopy; c += 32) {
        const bool is_rh = c < nrh;
        const int r = is_rh ? c : c - nrh;
        int row = j0 - 1 + r;
        row = row < 0 ? row + ny : (row >= ny ? row - ny : row);  // wrapped (finite data also at walls)
        const size_t src = ((size_t)kk * ny + row) * nx + (is_rh ? 0 : ocol);
        const uint32_t dst = smem_addr(slot + (is_rh ? L.rh + r * nx : L.xo + r * hx));
        bulk_load(dst, (is_rh ? a.rh : a.x) + src, 4u * (uint32_t)(is_rh ? nx : hx), bar);
    }
}

template <int N>
__device__ __forceinline__ void lds(float (&d)[N], const float* p) {
#pragma unroll
    for (int h = 0; h < N / 4; ++h) {
        const float4 v = *reinterpret_cast<const float4*>(p + 4 * h);
        d[4 * h] = v.x;
        d[4 * h + 1] = v.y;
        d[4 * h + 2] = v.z;
        d[4 * h + 3] = v.w;
    }
}

// Update the 4 cells of the updated colour at entries t0 .. t0+3 of row
// r (j = j0 + r) of plane k from the slots of planes k-1 (P), k (C), k+1 (Q);
// xu, F: the updated colour's x and f there.  Member M of each pair
// (2t + M) is updated; faces, neighbours and the order of every operation
// as in the register plane-tile kernel.
template <bool ZERO, bool XZ, int M>
__device__ __forceinline__ void update4(const StageArgs& a, const SlotLayout& L, const float* P, const float* C,
                                        const float* Q, int r, int j, int k, int t0, const float (&xu)[4],
                                        const float (&F)[4], float (&xn)[4]) {
    constexpr int V = 4;
    const int nx = L.nx, hx = L.hx;
    const float* rhr = C + L.rh + (r + 1) * nx;  // rho/2 of row j
    float R8[2 * V], Q8[2 * V];
    float rym[V], ryp[V], rzm[V], rzp[V];
    lds<2 * V>(R8, rhr + 2 * t0);
    lds<2 * V>(Q8, rhr - nx + 2 * t0);  // row j-1
#pragma unroll
    for (int v = 0; v < V; ++v) rym[v] = Q8[2 * v + M];
    lds<2 * V>(Q8, rhr + nx + 2 * t0);  // row j+1
#pragma unroll
    for (int v = 0; v < V; ++v) ryp[v] = Q8[2 * v + M];
    lds<2 * V>(Q8, P + L.rh + (r + 1) * nx + 2 * t0);  // plane k-1
#pragma unroll
    for (int v = 0; v < V; ++v) rzm[v] = Q8[2 * v + M];
    lds<2 * V>(Q8, Q + L.rh + (r + 1) * nx + 2 * t0);  // plane k+1
#pragma unroll
    for (int v = 0; v < V; ++v) rzp[v] = Q8[2 * v + M];
    // rho/2 of the x-neighbour outside the 8 cells: 2t0-1 (M = 0) or 2t0+8
    // (M = 1), wrapped around the row
    const float re = M == 0 ? rhr[t0 > 0 ? 2 * t0 - 1 : nx - 1] : rhr[t0 + V < hx ? 2 * t0 + 2 * V : 0];
    float xo[V], xym[V], xyp[V], xzm[V], xzp[V], xe = 0.f;
    if (ZERO) {
#pragma unroll
        for (int v = 0; v < V; ++v) xo[v] = xym[v] = xyp[v] = xzm[v] = xzp[v] = 0.f;
    } else {
        const float* xor_ = C + L.xo + (r + 1) * hx;
        lds<V>(xo, xor_ + t0);
        lds<V>(xym, xor_ - hx + t0);
        lds<V>(xyp, xor_ + hx + t0);
        lds<V>(xzm, P + L.xo + (r + 1) * hx + t0);
        lds<V>(xzp, Q + L.xo + (r + 1) * hx + t0);
        xe = M == 0 ? xor_[t0 > 0 ? t0 - 1 : hx - 1] : xor_[t0 + V < hx ? t0 + V : 0];
    }
    float vo[V], ro[V];
    if (M == 0) {
        vo[0] = xe;
        ro[0] = re;
#pragma unroll
        for (int v = 1; v < V; ++v) {
            vo[v] = xo[v - 1];
            ro[v] = R8[2 * v - 1];
        }
    } else {
#pragma unroll
        for (int v = 0; v < V - 1; ++v) {
            vo[v] = xo[v + 1];
            ro[v] = R8[2 * v + 2];
        }
        vo[V - 1] = xe;
        ro[V - 1] = re;
    }
    const bool ym_wall = a.g.wy && j == 0, yp_wall = a.g.wy && j == a.g.ny - 1;
    const bool zm_wall = a.g.wz && k == 0, zp_wall = a.g.wz && k == a.g.nz - 1;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const bool xwall = a.g.wx && (M == 0 ? (t0 + v == 0) : (t0 + v == hx - 1));
        const float ru = R8[2 * v + M], rin = R8[2 * v + 1 - M];
        const float b0 = xwall ? 0.f : bface(ru, ro[v]);
        const float b1 = bface(ru, rin);
        const float b2 = ym_wall ? 0.f : bface(ru, rym[v]);
        const float b3 = yp_wall ? 0.f : bface(ru, ryp[v]);
        const float b4 = zm_wall ? 0.f : bface(ru, rzm[v]);
        const float b5 = zp_wall ? 0.f : bface(ru, rzp[v]);
        const float w = rcp_approx(((b0 + b1) + (b2 + b3)) + (b4 + b5));
        const float fc = F[v] * a.h2;
        if (ZERO) {
            xn[v] = a.omega * w * fc;
        } else {
            const float x0 = XZ ? 0.f : xu[v];
            float acc = fmaf(b0, vo[v], fc);
            acc = fmaf(b1, xo[v], acc);
            acc = fmaf(b2, xym[v], acc);
            acc = fmaf(b3, xyp[v], acc);
            acc = fmaf(b4, xzm[v], acc);
            acc = fmaf(b5, xzp[v], acc);
            xn[v] = fmaf(a.omega, fmaf(w, acc, -x0), x0);
        }
    }
}

__device__ __forceinline__ void ldg4(float (&d)[4], const float* p) {
    const float4 v = __ldcs(reinterpret_cast<const float4*>(p));
    d[0] = v.x;
    d[1] = v.y;
    d[2] = v.z;
    d[3] = v.w;
}

// Grid: (ny / R tiles) x (zchunks), tile = blockIdx.x % tiles, so the CTAs
// running side by side hold adjacent tiles of the same planes and the halo
// rows one reads are the rows its neighbour reads at about the same time.
template <int R, bool ZERO, bool XZ>
__global__ void __launch_bounds__(R * 32) rbgs_rho_stage_kernel(StageArgs a) {
    extern __shared__ __align__(128) unsigned char stage_smem[];
    __shared__ __align__(8) unsigned long long bars[kStageSlots];
    __shared__ int abort_flag;
    const SlotLayout L = slot_layout(a.g.nx, R);
    float* slots = reinterpret_cast<float*>(stage_smem);
    const int nx = a.g.nx, hx = nx / 2, ny = a.g.ny, pl = nx * ny;
    const int ntiles = ny / R, npl = a.k1 - a.k0;
    const int tile = blockIdx.x % ntiles, zc = blockIdx.x / ntiles;
    const int ks = a.k0 + (int)((int64_t)npl * zc / a.zchunks);
    const int ke = a.k0 + (int)((int64_t)npl * (zc + 1) / a.zchunks);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStageSlots; ++s) mbar_init(smem_addr(&bars[s]), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (ke <= ks) return;  // uniform per CTA
    const int r = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j0 = tile * R, j = j0 + r;
    const int P = ke - ks + 2;  // planes ks-1 .. ke
    auto slot_of = [&](int q) { return slots + (size_t)(q % kStageSlots) * L.floats; };
    auto bar_of = [&](int q) { return smem_addr(&bars[q % kStageSlots]); };
    if (threadIdx.x < 32)
        for (int q = 0; q < P && q < kStageSlots; ++q) issue_plane<R, ZERO>(a, L, slot_of(q), bar_of(q), j0, ks - 1 + q);
    int issued = P < kStageSlots ? P : kStageSlots;
    const int ucol = a.col ? hx : 0;
    for (int q = 1; q <= P - 2; ++q) {
        const int k = ks - 1 + q;
        const int rb = k * pl + j * nx + ucol;  // the updated colour's half-row of row j
        // this plane's own values, read once: into registers before the waits
        float xu[2][4], F[2][4];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int t0 = 4 * lane + 128 * c;
            if (t0 < hx) {
                ldg4(F[c], a.f + rb + t0);
                if (!ZERO && !XZ) ldg4(xu[c], a.x + rb + t0);
            }
        }
        bool ok = true;
        for (int d = -1; d <= 1; ++d) {
            const int p = q + d;
            ok = ok && mbar_wait(bar_of(p), (uint32_t)((p / kStageSlots) & 1));
        }
        if (!ok) abort_flag = 1;
        if (ok) {
            const float* Ps = slot_of(q - 1);
            const float* Cs = slot_of(q);
            const float* Qs = slot_of(q + 1);
            const bool m0 = ((j + k + a.col) & 1) == 0;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int t0 = 4 * lane + 128 * c;
                if (t0 < hx) {
                    float xn[4];
                    if (m0)
                        update4<ZERO, XZ, 0>(a, L, Ps, Cs, Qs, r, j, k, t0, xu[c], F[c], xn);
                    else
                        update4<ZERO, XZ, 1>(a, L, Ps, Cs, Qs, r, j, k, t0, xu[c], F[c], xn);
                    __stcs(reinterpret_cast<float4*>(a.x + rb + t0), make_float4(xn[0], xn[1], xn[2], xn[3]));
                }
            }
            for (int t0 = 4 * lane + 256; t0 < hx; t0 += 128) {  // rows longer than 256 entries
                float xv[4], fv[4], xn[4];
                ldg4(fv, a.f + rb + t0);
                if (!ZERO && !XZ) ldg4(xv, a.x + rb + t0);
                if (m0)
                    update4<ZERO, XZ, 0>(a, L, Ps, Cs, Qs, r, j, k, t0, xv, fv, xn);
                else
                    update4<ZERO, XZ, 1>(a, L, Ps, Cs, Qs, r, j, k, t0, xv, fv, xn);
                __stcs(reinterpret_cast<float4*>(a.x + rb + t0), make_float4(xn[0], xn[1], xn[2], xn[3]));
            }
        }
        __syncthreads();  // every warp is done with slot q-1
        if (abort_flag) {
            // drain: this CTA's copies still in flight land before it exits
            if (threadIdx.x == 0) {
                atomicOr(a.fail, 1u);
                for (int p = q - 1; p < issued; ++p) mbar_wait(bar_of(p), (uint32_t)((p / kStageSlots) & 1));
            }
            __syncthreads();
            return;
        }
        const int qn = q - 1 + kStageSlots;  // the plane that reuses the released slot
        if (qn < P) {
            if (threadIdx.x < 32) issue_plane<R, ZERO>(a, L, slot_of(qn), bar_of(qn), j0, ks - 1 + qn);
            issued = qn + 1;
        }
    }
}

template <int R, bool ZERO, bool XZ>
cudaError_t launch_stage(StageArgs a, cudaStream_t st) {
    const SlotLayout L = slot_layout(a.g.nx, R);
    const size_t smem = (size_t)kStageSlots * L.floats * sizeof(float);
    auto kern = rbgs_rho_stage_kernel<R, ZERO, XZ>;
    static size_t set_for = 0;
    if (smem > set_for) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        set_for = smem;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, R * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int ntiles = a.g.ny / R, npl = a.k1 - a.k0;
    // as many z-chunks per tile as the resident CTAs allow, at least one plane each
    int z = (int)std::max<int64_t>(1, (int64_t)device_sms() * per_sm / ntiles);
    a.zchunks = std::min(z, npl);
    kern<<<(unsigned)(ntiles * a.zchunks), R * 32, smem, st>>>(a);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

// The staged pass needs: nx a multiple of 8 (16-byte rows and half-rows),
// ny a multiple of the tile height, a ring that fits in shared memory, and
// the 32-bit offsets of the level-0 kernels.
bool rho0_stage_fits(const Geo& g) {
    if (g.nx % 8 != 0 || g.ny % kStageRows != 0 || g.nz < 2) return false;
    const SlotLayout L = slot_layout(g.nx, kStageRows);
    return (size_t)kStageSlots * L.floats * sizeof(float) <= 200 * 1024;
}

cudaError_t launch_rbgs_rho_stage(const Geo& g, const float* rh, double h, const float* f, float* x, int color,
                                  double omega, bool zero_init, bool own_zero, int k0, int k1, unsigned* fail,
                                  cudaStream_t st) {
    StageArgs a{g, rh, f, x, (float)(h * h), (float)omega, color, k0, k1 < 0 ? g.nz : k1, 1, fail};
    if (zero_init) return launch_stage<kStageRows, true, false>(a, st);
    if (own_zero) return launch_stage<kStageRows, false, true>(a, st);
    return launch_stage<kStageRows, false, false>(a, st);
}

}  // namespace paris
