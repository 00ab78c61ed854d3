// TMA building blocks of the fused red-black SOR sweep (Sec. 2.6) shared by
// the single-domain kernels (les_sor_tma.cu) and the ensemble's persistent
// solve (les_kernels.cu): PTX wrappers for mbarriers and tiled bulk-tensor
// copies, the periodic images of halo cells, the block tile layout and the
// sweep of one 28 x BY x BZ block.
#pragma once

#include "les_internal.cuh"

#include <type_traits>

namespace les {
namespace tma {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

constexpr uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

// periodic image of (i, j, k): false when no periodic axis wraps; otherwise
// q = padded index of the image, or -1 when a non-periodic coordinate lies
// outside the padded box (the copy's zero fill)
__device__ __forceinline__ bool periodic_image(const Dom& d, int i, int j, int k, long long& q) {
    bool w = false;
    if (d.perx && (i < 1 || i > d.nx)) { i = ((i - 1) % d.nx + d.nx) % d.nx + 1; w = true; }
    if (d.pery && (j < 1 || j > d.ny)) { j = ((j - 1) % d.ny + d.ny) % d.ny + 1; w = true; }
    if (d.perz && (k < 1 || k > d.nz)) { k = ((k - 1) % d.nz + d.nz) % d.nz + 1; w = true; }
    if (!w) return false;
    q = (i < 0 || i > d.nx + 1 || j < 0 || j > d.ny + 1 || k < 0 || k > d.nz + 1) ? -1ll : d.at(i, j, k);
    return true;
}

// plane whose coefficients a ring plane takes: wrapped on a periodic z axis,
// else clamped to the padded range
__device__ __forceinline__ int coef_plane(const Dom& d, int k) {
    if (d.perz && (k < 1 || k > d.nz)) return ((k - 1) % d.nz + d.nz) % d.nz + 1;
    return min(max(k, 0), d.nz + 1);
}

template <int BY, int BZ>
struct TmaTile {
    static constexpr int BX = 28, DXW = 36, FXW = 48;
    static constexpr int DY = BY + 4, DZ = BZ + 4, RY = BY + 2, RZ = BZ + 2;
    static constexpr uint32_t BYTES_D = DXW * DY * DZ * 4;
    static constexpr uint32_t BYTES_R = DXW * RY * RZ * 4;
    static constexpr uint32_t BYTES_F = FXW * RY * RZ;
    static constexpr uint32_t OFF_R = align_up(BYTES_D, 128);
    static constexpr uint32_t OFF_F = OFF_R + align_up(BYTES_R, 128);
    static constexpr uint32_t OFF_CN = OFF_F + align_up(BYTES_F, 128);
    static constexpr uint32_t OFF_CT = OFF_CN + RZ * 64 * 4;
    static constexpr uint32_t OFF_T4 = align_up(OFF_CT + 2 * RZ * 4, 16);   // float4 [64]: ae, aw, an, as
    static constexpr uint32_t OFF_BAR = OFF_T4 + 64 * 16;
    static constexpr uint32_t SMEM = OFF_BAR + 8;
};

// One block (bx, by, bz) of the fused sweep on the CTA's shared memory sm,
// whose mbarrier (initialised by the caller) completes phase `phase` when the
// block's copies have landed.  Returns false after recording a timed-out
// wait.  The caller separates two blocks on one CTA by a barrier.
template <int BY, int BZ, int NT>
__device__ __forceinline__ bool sor_tma_block(unsigned char* sm, const CUtensorMap* td, const CUtensorMap* tr,
                                              const CUtensorMap* tf, const Geo<float>& g,
                                              const float* __restrict__ din, const float* __restrict__ rin,
                                              float* __restrict__ dout, bool zero_start, Scalars* __restrict__ sc,
                                              int bx, int by, int bz, uint32_t phase) {
    using TT = TmaTile<BY, BZ>;
    constexpr int BX = TT::BX, DXW = TT::DXW, FXW = TT::FXW, DY = TT::DY, RY = TT::RY, RZ = TT::RZ;
    float(*sD)[DY][DXW] = reinterpret_cast<float(*)[DY][DXW]>(sm);
    float(*sR)[RY][DXW] = reinterpret_cast<float(*)[RY][DXW]>(sm + TT::OFF_R);
    uint8_t(*sF)[RY][FXW] = reinterpret_cast<uint8_t(*)[RY][FXW]>(sm + TT::OFF_F);
    float(*sCN)[64] = reinterpret_cast<float(*)[64]>(sm + TT::OFF_CN);
    float* sCT = reinterpret_cast<float*>(sm + TT::OFF_CT);
    float* sCB = sCT + RZ;
    const Dom& d = g.d;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y, lane = tid & 31, warp = tid >> 5;   // 1-D or 32 x 8
    constexpr int NW = NT / 32;
    const int i0 = 1 + bx * BX, j0 = 1 + by * BY, k0 = 1 + bz * BZ;
    const int xd = bx * BX;                   // padded column of i0 - 4
    const int xf = xd & ~15, off = xd - xf;
    const uint32_t bar = smem_u32(sm + TT::OFF_BAR);
    if (tid == 0) {
        mbar_expect_tx(bar, TT::BYTES_R + TT::BYTES_F + (zero_start ? 0u : TT::BYTES_D));
        if (!zero_start) tma_load_3d(smem_u32(sD), td, xd, j0 - 2, k0 - 2, bar);
        tma_load_3d(smem_u32(sR), tr, xd, j0 - 1, k0 - 1, bar);
        tma_load_3d(smem_u32(sF), tf, xf, j0 - 1, k0 - 1, bar);
    }
    // per-plane coefficients and the block's rows of the cn1 table while the copies fly
    for (int q = tid; q < RZ * 64; q += NT) {
        const int kk = q >> 6, m = q & 63;
        const int k = coef_plane(d, k0 - 1 + kk);
        sCN[kk][m] = g.cn1[k * 64 + m];
        if (m == 0) {
            const float ct = g.cT[k], cb = g.cB[k];
            sCT[kk] = ct;
            sCB[kk] = cb;
        }
    }
    if (zero_start) {
        float* p = &sD[0][0][0];
        for (int q = tid; q < DXW * DY * TT::DZ; q += NT) p[q] = 0.f;
    }
    if (tid < 64) {
        const float cx = g.cx, cy = g.cy;
        reinterpret_cast<float4*>(sm + TT::OFF_T4)[tid] =
            make_float4((tid & F_E) ? cx : 0.f, (tid & F_W) ? cx : 0.f, (tid & F_N) ? cy : 0.f, (tid & F_S) ? cy : 0.f);
    }
    __syncthreads();
    bool ok = false;
    const uint64_t t0 = global_ns();
    while (!(ok = mbar_try_wait(bar, phase)))
        if (global_ns() - t0 > 1000000000ull) break;
    if (!__syncthreads_and(ok)) {
        if (tid == 0) atomicExch(&sc->timeout, 1);
        const uint64_t t1 = global_ns();     // give copies still in flight a bounded chance to land
        while (!mbar_try_wait(bar, phase))
            if (global_ns() - t1 > 1000000000ull) break;
        return false;
    }
    if ((d.perx && (i0 - 2 < 1 || i0 + BX + 1 > d.nx)) || (d.pery && (j0 - 2 < 1 || j0 + BY + 1 > d.ny)) ||
        (d.perz && (k0 - 2 < 1 || k0 + BZ + 1 > d.nz))) {
        // halo across a periodic face: the images of the cells the sweep reads
        // (d on i0-2 .. i0+BX+1 with a 2-cell halo in j, k; r and flags on the
        // block + 1 ring)
        if (!zero_start)
            for (int q = tid; q < TT::DZ * DY * (BX + 4); q += NT) {
                const int x = 2 + q % (BX + 4), y = (q / (BX + 4)) % DY, z = q / ((BX + 4) * DY);
                long long s;
                if (periodic_image(d, i0 - 4 + x, j0 - 2 + y, k0 - 2 + z, s)) sD[z][y][x] = s >= 0 ? din[s] : 0.f;
            }
        for (int q = tid; q < RZ * RY * (BX + 2); q += NT) {
            const int x = q % (BX + 2), y = (q / (BX + 2)) % RY, z = q / ((BX + 2) * RY);
            long long s;
            if (periodic_image(d, i0 - 1 + x, j0 - 1 + y, k0 - 1 + z, s)) {
                sR[z][y][x + 3] = s >= 0 ? rin[s] : 0.f;
                sF[z][y][x + 3 + off] = s >= 0 ? g.flags[s] : (uint8_t)0;
            }
        }
        __syncthreads();
    }
    const float omega = g.omega;
    const float4* T4 = reinterpret_cast<const float4*>(sm + TT::OFF_T4);
    // the update of Sec. 2.6 at shared cell p (plane row kz of the block's
    // coefficient rows), branch-free: the in-plane coefficients of the
    // cell's open-face mask from T4, the vertical ones selected by the mask
    auto relax = [&](float* p, int kz, uint8_t f, float rhs) {
        constexpr int PZ = DY * DXW;
        const float4 a = T4[f & 63];
        const float cn1 = sCN[kz][f & 63];
        const float at = (f & F_T) ? sCT[kz] : 0.f, ab = (f & F_B) ? sCB[kz] : 0.f;
        float s = 0.f;
        s += a.x * p[1];
        s += a.y * p[-1];
        s += a.z * p[DXW];
        s += a.w * p[-DXW];
        s += at * p[PZ];
        s += ab * p[-PZ];
        float own = p[0];
        float reltmp = omega * (cn1 * (s - rhs) - own);
        p[0] = own + reltmp;
    };
    float* const D0 = &sD[0][0][0];
    const float* const R0 = &sR[0][0][0];
    const uint8_t* const F0 = &sF[0][0][0];
    const int half = lane >> 4, m = lane & 15;
    const int par0 = (i0 + j0 + k0) & 1;
    // red (i+j+k odd) on the block + 1 ring (i0-1 .. i0+28): 15 per row, two rows per warp pass
    if (m < (BX + 2) / 2)
        for (int p = warp; 2 * p < RY * RZ; p += NW) {
            const int rw = 2 * p + half;
            if (rw >= RY * RZ) break;
            const int jj = rw % RY, kk = rw / RY;
            const int ii = 2 * m + ((par0 + jj + kk) & 1);                   // i = i0 - 1 + ii
            const uint8_t f = F0[(kk * RY + jj) * FXW + ii + 3 + off];
            if (f & F_UNK)
                relax(D0 + ((kk + 1) * DY + jj + 1) * DXW + ii + 3, kk, f, R0[(kk * RY + jj) * DXW + ii + 3]);
        }
    __syncthreads();
    // black (i+j+k even) on the block (i0 .. i0+27): 14 per row
    if (m < BX / 2)
        for (int p = warp; 2 * p < BY * BZ; p += NW) {
            const int rw = 2 * p + half;
            if (rw >= BY * BZ) break;
            const int jj = rw % BY, kk = rw / BY;
            const int ii = 2 * m + ((par0 + jj + kk) & 1);                   // i = i0 + ii
            const uint8_t f = F0[((kk + 1) * RY + jj + 1) * FXW + ii + 4 + off];
            if (f & F_UNK)
                relax(D0 + ((kk + 2) * DY + jj + 2) * DXW + ii + 4, kk + 1, f,
                      R0[((kk + 1) * RY + jj + 1) * DXW + ii + 4]);
        }
    __syncthreads();
    // store the block (cells that are not unknowns hold 0 in d and in the
    // tile): 4 rows per warp pass, 7 lanes x 4 cells (16-byte aligned) per row
    {
        const int c = lane & 7, sub = lane >> 3;
        const int i = i0 + 4 * c;
        const int kend = min(BZ, d.nz + 1 - k0), jend = min(BY, d.ny + 1 - j0);
        if (c < BX / 4 && i <= d.nx)
            for (int rw = 4 * warp + sub; rw < BY * BZ; rw += 4 * NW) {
                const int jj = rw % BY, kk = rw / BY;
                if (jj >= jend || kk >= kend) continue;
                const float4 v = *reinterpret_cast<const float4*>(D0 + ((kk + 2) * DY + jj + 2) * DXW + 4 + 4 * c);
                float* o = dout + d.at(i, j0 + jj, k0 + kk);
                if (i + 3 <= d.nx) {
                    *reinterpret_cast<float4*>(o) = v;
                } else {
                    o[0] = v.x;
                    if (i + 1 <= d.nx) o[1] = v.y;
                    if (i + 2 <= d.nx) o[2] = v.z;
                }
            }
    }
    return true;
}


// Shared-memory accesses at a 32-bit shared address plus a compile-time byte
// offset (one instruction each, the offset in the instruction's immediate).
template <int OFF>
__device__ __forceinline__ float lds_f32(uint32_t a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(a), "n"(OFF) : "memory");
    return v;
}
template <int OFF>
__device__ __forceinline__ uint32_t lds_u8(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u8 %0, [%1+%2];" : "=r"(v) : "r"(a), "n"(OFF) : "memory");
    return v;
}
template <int OFF>
__device__ __forceinline__ float2 lds_f32x2(uint32_t a) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2+%3];" : "=f"(v.x), "=f"(v.y) : "r"(a), "n"(OFF) : "memory");
    return v;
}
// store v at a + OFF when pred != 0
template <int OFF>
__device__ __forceinline__ void sts_f32_if(uint32_t a, float v, uint32_t pred) {
    asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %2, 0;\n @p st.shared.f32 [%0+%3], %1;\n}\n" ::"r"(a), "f"(v),
                 "r"(pred), "n"(OFF)
                 : "memory");
}

// Untiled bulk copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) from global memory into shared memory, completing on mbarrier bar.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// Rows of the per-plane coefficient table of the column-walk sweeps: for
// padded plane k, cn1 over the 64 open-face masks, then cT, cB and two pad
// floats (272 bytes).  The table has kColTableRows rows past plane nz + 1, so a
// block near the top copies whole rows; ring planes across a periodic z face
// hold the wrapped plane's values, other planes outside 0 .. nz + 1 the
// nearest one's.
constexpr int kColRow = 68;

// One lane's walk up a column of one colour (NP updates, planes kk0, kk0+2,
// ...) in the column-walk block sweep.  Shared addresses: ad = d cell one
// plane below the first update, ar / af = its r / flag cell, acn = the
// coefficient row of plane kk0.  PZ, PR, PF: plane strides of the d, r and
// flag tiles (elements); DXW: row stride of d and r.  The next update's
// loads are issued before this update's store; none of them reads a cell
// the walk writes (the neighbours have the other colour).
struct ColVals {
    uint32_t fl;
    float rhs, up, ve, vw, vn, vs, own, cn1;
};
template <int NP, int PZ, int PR, int PF, int DXW>
struct ColWalk {
    static constexpr int RB = kColRow * 4;        // bytes per coefficient row
    uint32_t ad, ar, af, acn;
    float cx, cy, omega;
    template <int T>
    __device__ __forceinline__ void load(ColVals& v) const {
        constexpr int OD = 2 * T * PZ * 4;
        v.fl = lds_u8<2 * T * PF>(af);
        v.rhs = lds_f32<2 * T * PR * 4>(ar);
        v.up = lds_f32<OD + 2 * PZ * 4>(ad);
        v.ve = lds_f32<OD + (PZ + 1) * 4>(ad);
        v.vw = lds_f32<OD + (PZ - 1) * 4>(ad);
        v.vn = lds_f32<OD + (PZ + DXW) * 4>(ad);
        v.vs = lds_f32<OD + (PZ - DXW) * 4>(ad);
        v.own = lds_f32<OD + PZ * 4>(ad);
        v.cn1 = lds_f32<2 * T * RB>(acn + ((v.fl & 63u) << 2));
    }
    template <int T>
    __device__ __forceinline__ void step(ColVals& cur, float& lo) const {
        ColVals nx{};
        if constexpr (T + 1 < NP) load<T + 1>(nx);
        const float2 cv = lds_f32x2<2 * T * RB + 256>(acn);
        float s = 0.f;
        s += cx * cur.ve;
        s += cx * cur.vw;
        s += cy * cur.vn;
        s += cy * cur.vs;
        s += cv.x * cur.up;
        s += cv.y * lo;
        float reltmp = omega * (cur.cn1 * (s - cur.rhs) - cur.own);
        sts_f32_if<2 * T * PZ * 4 + PZ * 4>(ad, cur.own + reltmp, cur.fl & F_UNK);
        lo = cur.up;
        cur = nx;
    }
    template <int... T>
    __device__ __forceinline__ void run(std::integer_sequence<int, T...>) const {
        float lo = lds_f32<0>(ad);
        ColVals cur;
        load<0>(cur);
        (step<T>(cur, lo), ...);
    }
    __device__ __forceinline__ void operator()() const { run(std::make_integer_sequence<int, NP>{}); }
};

// Shared memory of the column-walk sweep: the d, r and flag tiles of
// TmaTile, then the block's RZ rows of the coefficient table (kColRow floats
// each), then the mbarrier.
template <int BY, int BZ>
struct ColTile {
    using TT = TmaTile<BY, BZ>;
    static constexpr int RZ = TT::RZ;
    static_assert(BZ <= kColTableRows, "the coefficient table is padded for BZ <= kColTableRows");
    static constexpr uint32_t OFF_TAB = TT::OFF_CN;                   // 128-byte aligned
    static constexpr uint32_t BYTES_TAB = RZ * kColRow * 4;
    static constexpr uint32_t STAGE = align_up(OFF_TAB + BYTES_TAB, 128);
    static constexpr uint32_t SMEM = STAGE + 8;                       // the stage + its mbarrier
};

// The copies of block (bx, by, bz) into stage st on mbarrier bar (one
// thread): col_expect arms the barrier for all of them, col_issue_static
// copies what no sweep writes (r and the flags with a 1-cell ring, the
// block's coefficient rows), col_issue_d the correction d with a 2-cell halo
// (skipped when the sweep starts from zero).
template <int BY, int BZ>
__device__ __forceinline__ void col_expect(uint32_t bar, bool zero_start) {
    using TT = TmaTile<BY, BZ>;
    mbar_expect_tx(bar, TT::BYTES_R + TT::BYTES_F + ColTile<BY, BZ>::BYTES_TAB + (zero_start ? 0u : TT::BYTES_D));
}
// the constant part (flags and coefficient rows: no kernel of a solve writes
// them) and r (written only between batches of sweeps)
template <int BY, int BZ>
__device__ __forceinline__ void col_issue_const(unsigned char* st, uint32_t bar, const CUtensorMap* tf,
                                                const float* ctab, int bx, int by, int bz) {
    using TT = TmaTile<BY, BZ>;
    const int xf = (bx * TT::BX) & ~15, j0 = 1 + by * BY, k0 = 1 + bz * BZ;
    tma_load_3d(smem_u32(st + TT::OFF_F), tf, xf, j0 - 1, k0 - 1, bar);
    bulk_load(smem_u32(st + ColTile<BY, BZ>::OFF_TAB), ctab + (size_t)(k0 - 1) * kColRow, ColTile<BY, BZ>::BYTES_TAB,
              bar);
}
template <int BY, int BZ>
__device__ __forceinline__ void col_issue_r(unsigned char* st, uint32_t bar, const CUtensorMap* tr, int bx, int by,
                                            int bz) {
    using TT = TmaTile<BY, BZ>;
    tma_load_3d(smem_u32(st + TT::OFF_R), tr, bx * TT::BX, 1 + by * BY - 1, 1 + bz * BZ - 1, bar);
}
template <int BY, int BZ>
__device__ __forceinline__ void col_issue_static(unsigned char* st, uint32_t bar, const CUtensorMap* tr,
                                                 const CUtensorMap* tf, const float* ctab, int bx, int by, int bz) {
    col_issue_r<BY, BZ>(st, bar, tr, bx, by, bz);
    col_issue_const<BY, BZ>(st, bar, tf, ctab, bx, by, bz);
}
// expected bytes without an arrival (the arrival comes with a later
// arrive.expect_tx of the remaining bytes)
__device__ __forceinline__ void mbar_expect_tx_only(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
template <int BY, int BZ>
__device__ __forceinline__ void col_issue_d(unsigned char* st, uint32_t bar, const CUtensorMap* td, int bx, int by,
                                            int bz) {
    tma_load_3d(smem_u32(st), td, bx * TmaTile<BY, BZ>::BX, 1 + by * BY - 2, 1 + bz * BZ - 2, bar);
}
template <int BY, int BZ>
__device__ __forceinline__ void col_issue(unsigned char* st, uint32_t bar, const CUtensorMap* td, const CUtensorMap* tr,
                                          const CUtensorMap* tf, const float* ctab, int bx, int by, int bz,
                                          bool zero_start) {
    col_expect<BY, BZ>(bar, zero_start);
    if (!zero_start) col_issue_d<BY, BZ>(st, bar, td, bx, by, bz);
    col_issue_static<BY, BZ>(st, bar, tr, tf, ctab, bx, by, bz);
}

// After the copies of block (bx, by, bz) have landed in stage st: zero the d
// tile on a zero start, the periodic halo images (a warp per tile row; rows
// that cross no periodic y or z face are skipped whole unless the block
// touches a periodic x face), red on the block + ring, black on the block.
// Ends with a CTA barrier.
template <int BY, int BZ, int NT>
__device__ __forceinline__ void col_relax(unsigned char* st, const Geo<float>& g, const float* __restrict__ din,
                                          const float* __restrict__ rin, bool zero_start, int bx, int by, int bz) {
    using TT = TmaTile<BY, BZ>;
    using CT = ColTile<BY, BZ>;
    constexpr int BX = TT::BX, DXW = TT::DXW, FXW = TT::FXW, DY = TT::DY, DZ = TT::DZ, RY = TT::RY, RZ = TT::RZ;
    constexpr int PZ = DY * DXW, PR = RY * DXW, PF = RY * FXW;
    constexpr int NW = NT / 32;
    static_assert(BY % 2 == 0 && BZ % 2 == 0, "the column walk pairs rows and planes");
    const Dom& d = g.d;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y, lane = tid & 31, warp = tid >> 5;   // 1-D or 32 x 8
    const int i0 = 1 + bx * BX, j0 = 1 + by * BY, k0 = 1 + bz * BZ;
    const int xd = bx * BX, off = xd - (xd & ~15);
    float* const D0 = reinterpret_cast<float*>(st);
    if (zero_start) {
        for (int q = tid; q < DXW * DY * DZ / 4; q += NT) reinterpret_cast<float4*>(D0)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
    }
    const bool wx = d.perx && (i0 - 2 < 1 || i0 + BX + 1 > d.nx);
    if (wx || (d.pery && (j0 - 2 < 1 || j0 + BY + 1 > d.ny)) || (d.perz && (k0 - 2 < 1 || k0 + BZ + 1 > d.nz))) {
        float(*sD)[DY][DXW] = reinterpret_cast<float(*)[DY][DXW]>(st);
        float(*sR)[RY][DXW] = reinterpret_cast<float(*)[RY][DXW]>(st + TT::OFF_R);
        uint8_t(*sF)[RY][FXW] = reinterpret_cast<uint8_t(*)[RY][FXW]>(st + TT::OFF_F);
        auto row_wraps = [&](int j, int k) {
            return wx || (d.pery && (j < 1 || j > d.ny)) || (d.perz && (k < 1 || k > d.nz));
        };
        if (!zero_start)
            for (int rw = warp; rw < DZ * DY; rw += NW) {
                const int y = rw % DY, z = rw / DY;
                if (!row_wraps(j0 - 2 + y, k0 - 2 + z)) continue;
                for (int x = 2 + lane; x < BX + 6; x += 32) {
                    long long s;
                    if (periodic_image(d, i0 - 4 + x, j0 - 2 + y, k0 - 2 + z, s)) sD[z][y][x] = s >= 0 ? din[s] : 0.f;
                }
            }
        for (int rw = warp; rw < RZ * RY; rw += NW) {
            const int y = rw % RY, z = rw / RY;
            if (!row_wraps(j0 - 1 + y, k0 - 1 + z)) continue;
            for (int x = lane; x < BX + 2; x += 32) {
                long long s;
                if (periodic_image(d, i0 - 1 + x, j0 - 1 + y, k0 - 1 + z, s)) {
                    sR[z][y][x + 3] = s >= 0 ? rin[s] : 0.f;
                    sF[z][y][x + 3 + off] = s >= 0 ? g.flags[s] : (uint8_t)0;
                }
            }
        }
        __syncthreads();
    }
    const float omega = g.omega, cx = g.cx, cy = g.cy;
    const int half = lane >> 4, m = lane & 15;
    const int par0 = (i0 + j0 + k0) & 1;
    const uint32_t sD0 = smem_u32(st), sR0 = smem_u32(st + TT::OFF_R), sF0 = smem_u32(st + TT::OFF_F);
    const uint32_t sT0 = smem_u32(st + CT::OFF_TAB);
    constexpr uint32_t RB = kColRow * 4;
    // red (i+j+k odd) on the block + ring: task = (row pair, plane parity);
    // the lane's d cell one plane below its first update is (kp, jj+1, ii+3)
    if (m < (BX + 2) / 2)
        for (int task = warp; task < RY; task += NW) {
            const int kp = task & 1, jj = (task >> 1) * 2 + half;
            const int ii = 2 * m + ((par0 + jj + kp) & 1);                  // i = i0 - 1 + ii
            const ColWalk<RZ / 2, PZ, PR, PF, DXW> w{sD0 + 4u * ((kp * DY + jj + 1) * DXW + ii + 3),
                                                     sR0 + 4u * ((kp * RY + jj) * DXW + ii + 3),
                                                     sF0 + (uint32_t)((kp * RY + jj) * FXW + ii + 3 + off),
                                                     sT0 + RB * kp, cx, cy, omega};
            w();
        }
    __syncthreads();
    // black (i+j+k even) on the block: one plane below the first update is
    // d cell (kp+1, jj+2, ii+4)
    if (m < BX / 2)
        for (int task = warp; task < BY; task += NW) {
            const int kp = task & 1, jj = (task >> 1) * 2 + half;
            const int ii = 2 * m + ((par0 + jj + kp) & 1);                  // i = i0 + ii
            const ColWalk<BZ / 2, PZ, PR, PF, DXW> w{sD0 + 4u * (((kp + 1) * DY + jj + 2) * DXW + ii + 4),
                                                     sR0 + 4u * (((kp + 1) * RY + jj + 1) * DXW + ii + 4),
                                                     sF0 + (uint32_t)(((kp + 1) * RY + jj + 1) * FXW + ii + 4 + off),
                                                     sT0 + RB * (kp + 1), cx, cy, omega};
            w();
        }
    __syncthreads();
}

// Store block (bx, by, bz) of stage st (cells that are not unknowns hold 0
// in d and in the tile): 4 rows per warp pass, 7 lanes x 4 cells (16-byte
// aligned) per row.
template <int BY, int BZ, int NT>
__device__ __forceinline__ void col_store(const unsigned char* st, const Dom& d, float* __restrict__ dout, int bx, int by,
                                          int bz) {
    using TT = TmaTile<BY, BZ>;
    constexpr int BX = TT::BX, DXW = TT::DXW, DY = TT::DY, NW = NT / 32;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y, lane = tid & 31, warp = tid >> 5;
    const int i0 = 1 + bx * BX, j0 = 1 + by * BY, k0 = 1 + bz * BZ;
    const float* D0 = reinterpret_cast<const float*>(st);
    const int c = lane & 7, sub = lane >> 3;
    const int i = i0 + 4 * c;
    const int kend = min(BZ, d.nz + 1 - k0), jend = min(BY, d.ny + 1 - j0);
    // rows rw = r0, r0 + 4 NW, ...: with BY | 4 NW the row jj stays and the
    // plane kk advances by 4 NW / BY per pass
    static_assert((4 * NW) % BY == 0, "store passes keep the row");
    constexpr int DK = 4 * NW / BY;
    const int r0 = 4 * warp + sub, jj = r0 % BY;
    if (c < BX / 4 && i <= d.nx && jj < jend) {
        const float* src = D0 + ((r0 / BY + 2) * DY + jj + 2) * DXW + 4 + 4 * c;
        float* o = dout + d.at(i, j0 + jj, k0 + r0 / BY);
        const bool full = i + 3 <= d.nx;
        for (int kk = r0 / BY; kk < kend; kk += DK, src += DK * DY * DXW, o += DK * d.plane) {
            const float4 v = *reinterpret_cast<const float4*>(src);
            if (full) {
                *reinterpret_cast<float4*>(o) = v;
            } else {
                o[0] = v.x;
                if (i + 1 <= d.nx) o[1] = v.y;
                if (i + 2 <= d.nx) o[2] = v.z;
            }
        }
    }
}

// Bounded wait (1 s) of one thread for phase `phase` of mbarrier bar.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase) {
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, phase))
        if (global_ns() - t0 > 1000000000ull) return false;
    return true;
}

// The rest of the column-walk block sweep once the block's copies are
// issued on the stage's mbarrier: the bounded wait, the relaxation and the
// store.  Returns false after recording a timed-out wait.
template <int BY, int BZ, int NT>
__device__ __forceinline__ bool sor_col_finish(unsigned char* sm, const Geo<float>& g, const float* __restrict__ din,
                                               const float* __restrict__ rin, float* __restrict__ dout,
                                               bool zero_start, Scalars* __restrict__ sc, int bx, int by, int bz,
                                               uint32_t phase) {
    const uint32_t bar = smem_u32(sm + ColTile<BY, BZ>::STAGE);
    const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
    bool ok = true;
    if (lead) ok = mbar_wait_bounded(bar, phase);
    if (!__syncthreads_and(ok)) {
        if (lead) {
            atomicExch(&sc->timeout, 1);
            mbar_wait_bounded(bar, phase);     // give copies still in flight a bounded chance to land
        }
        __syncthreads();
        return false;
    }
    col_relax<BY, BZ, NT>(sm, g, din, rin, zero_start, bx, by, bz);
    col_store<BY, BZ, NT>(sm, g.d, dout, bx, by, bz);
    return true;
}

// The block sweep of sor_tma_block with fewer instructions per cell.  It
// relies on the correction being zero on every cell that is not an unknown
// (solid cells, ghost cells, padding; every kernel that writes d keeps it
// so), so a closed face contributes c * 0 whatever its coefficient: the six
// neighbour coefficients are the uniform cx, cx, cy, cy, cT(k), cB(k), and
// only cn1 depends on the open-face mask.  The products and sums are those
// of the masked update in the same order, so the iterate is the same.
//
// Work split: a warp relaxes two rows of one colour at every other plane,
// one row per half-warp and one lane per column (every other cell of the
// row), and each lane walks its column up the block; the cell below the
// next update is the one above the current update, so it stays in a
// register, and the plane (hence cT, cB and the cn1 row) is the same for
// the whole warp.  Red runs on the block + 1-cell ring (RY rows, RZ planes),
// black on the block (BY rows, BZ planes).  One thread polls the copies'
// mbarrier; the CTA barrier then passes their completion on to every thread.
template <int BY, int BZ, int NT>
__device__ __forceinline__ bool sor_col_block(unsigned char* sm, const CUtensorMap* td, const CUtensorMap* tr,
                                              const CUtensorMap* tf, const Geo<float>& g,
                                              const float* __restrict__ din, const float* __restrict__ rin,
                                              float* __restrict__ dout, bool zero_start, Scalars* __restrict__ sc,
                                              int bx, int by, int bz, uint32_t phase) {
    using CT = ColTile<BY, BZ>;
    const uint32_t bar = smem_u32(sm + CT::STAGE);
    const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
    if (lead) col_issue<BY, BZ>(sm, bar, td, tr, tf, g.ctab, bx, by, bz, zero_start);
    return sor_col_finish<BY, BZ, NT>(sm, g, din, rin, dout, zero_start, sc, bx, by, bz, phase);
}

}  // namespace tma
}  // namespace les
