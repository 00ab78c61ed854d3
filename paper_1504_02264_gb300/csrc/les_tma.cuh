// TMA building blocks of the fused red-black SOR sweep (Sec. 2.6) shared by
// the single-domain kernels (les_sor_tma.cu) and the ensemble's persistent
// solve (les_kernels.cu): PTX wrappers for mbarriers and tiled bulk-tensor
// copies, the periodic images of halo cells, the block tile layout and the
// sweep of one 28 x BY x BZ block.
#pragma once

#include "les_internal.cuh"

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


}  // namespace tma
}  // namespace les
