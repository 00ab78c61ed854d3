// TMA variant of the fused red-black SOR sweep (Sec. 2.6) for FP32 domains.
//
// A CTA owns a 28 x BY x BZ block.  One thread issues three tiled bulk-tensor
// copies (cp.async.bulk.tensor) into shared memory on one mbarrier: the
// correction d on the block plus a 2-cell halo, and r and the cell flags on
// the block plus a 1-cell ring.  Cells outside the padded array arrive as
// zeros (the copy's out-of-bounds fill), which is what the Neumann ghost
// layer holds, so no per-element bounds logic is needed.  While the copies
// are in flight the threads build the per-plane cn1 table.  Then red on the
// block + ring, black on the block, and the block is stored (unknowns only),
// exactly as in the other fused variants (bit-identical iterate).
//
// Periodic axes: a copy cannot wrap, so after the copies land the blocks
// whose halo crosses a periodic face overwrite the out-of-range cells of the
// tiles with plain loads of their periodic images (d, r and flags), and the
// ring planes take the coefficients of the wrapped plane.  Interior blocks
// skip this step.  The persistent double-buffered variant (k_sor_pipe) stays
// restricted to domains without periodic axes.
//
// Alignment: the d and r tiles start at padded column 28*bx (a multiple of 4
// floats = 16 bytes); the flag tile starts at the multiple of 16 bytes below it
// and is 48 bytes wide.  The wait on the mbarrier is bounded by the global
// timer; on a timeout the block records it in Scalars::timeout and returns
// without touching the output.
#include "les_internal.cuh"
#include "les_tma.cuh"

namespace les {
namespace {

using namespace tma;

template <int BY, int BZ, int NT>
__global__ void __launch_bounds__(NT)
k_sor_tma(const __grid_constant__ CUtensorMap td, const __grid_constant__ CUtensorMap tr,
          const __grid_constant__ CUtensorMap tf, Geo<float> g, const float* __restrict__ din,
          const float* __restrict__ rin, float* __restrict__ dout, int zero_arg, Scalars* __restrict__ sc) {
    extern __shared__ __align__(128) unsigned char sm[];
    pdl_wait();
    if (sc->done) return;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(sm + TmaTile<BY, BZ>::OFF_BAR), 1);
        mbar_fence_init();
    }
    __syncthreads();
    const bool zero_start = zero_arg == 1 || (zero_arg == 2 && sc->zflag);
    sor_tma_block<BY, BZ, NT>(sm, &td, &tr, &tf, g, din, rin, dout, zero_start, sc, blockIdx.x, blockIdx.y, blockIdx.z,
                              0u);
}

// The same block sweep with the column-walk update (sor_col_block): fewer
// instructions per cell for the same iterate.  The flags and coefficient
// rows (written by no kernel of a solve) are copied before the dependency
// wait.  pre = 1 when the kernel before it in the stream is a sweep of the
// same batch: sweeps write only d, so r is copied before the wait as well,
// and only d after it.  Each CTA lets the next kernel launch once
// its copies are issued (a dependent kernel waits for this grid to complete
// before it touches anything this sweep writes).
template <int BY, int BZ, int NT>
__global__ void __launch_bounds__(NT)
k_sor_col(const __grid_constant__ CUtensorMap td, const __grid_constant__ CUtensorMap tr,
          const __grid_constant__ CUtensorMap tf, Geo<float> g, const float* __restrict__ din,
          const float* __restrict__ rin, float* __restrict__ dout, int zero_arg, Scalars* __restrict__ sc, int pre) {
    using CT = ColTile<BY, BZ>;
    extern __shared__ __align__(128) unsigned char sm[];
    const uint32_t bar = smem_u32(sm + CT::STAGE);
    const bool lead = threadIdx.x == 0;
    const int bx = blockIdx.x, by = blockIdx.y, bz = blockIdx.z;
    using TT = TmaTile<BY, BZ>;
    if (lead) {
        mbar_init(bar, 1);
        mbar_fence_init();
        if (pre) {
            col_expect<BY, BZ>(bar, false);
            col_issue_static<BY, BZ>(sm, bar, &tr, &tf, g.ctab, bx, by, bz);
        } else {
            // the first sweep of a batch: only the constant tiles before the wait
            mbar_expect_tx_only(bar, TT::BYTES_F + CT::BYTES_TAB);
            col_issue_const<BY, BZ>(sm, bar, &tf, g.ctab, bx, by, bz);
        }
    }
    pdl_wait();
    const bool zero_start = !pre && (zero_arg == 1 || (zero_arg == 2 && sc->zflag));
    if (lead) {
        if (!pre) {
            mbar_expect_tx(bar, TT::BYTES_R + (zero_start ? 0u : TT::BYTES_D));
            col_issue_r<BY, BZ>(sm, bar, &tr, bx, by, bz);
        }
        if (!zero_start) col_issue_d<BY, BZ>(sm, bar, &td, bx, by, bz);
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (sc->done) {       // uniform over the grid: let the copies land (bounded), then leave
        if (lead) mbar_wait_bounded(bar, 0u);
        __syncthreads();
        return;
    }
    sor_col_finish<BY, BZ, NT>(sm, g, din, rin, dout, zero_start, sc, bx, by, bz, 0u);
}

// The batched sweep of an ensemble: persistent CTAs walk the flattened list
// of every member's 28 x BY x BZ blocks (member m owns items tbeg[m] ..
// tbeg[m+1]-1) and sweep each block of the members whose solve is still
// running, with the member's own tensor maps (four per member in global
// memory: d[0], d[1], r, flags) and arguments -- the column-walk block sweep
// of the single-domain kernel, so a member evolves as it would alone with
// tile 29.
// One launch per sweep covers every member.
template <int BY, int BZ, int NT>
__global__ void __launch_bounds__(NT)
k_sor_tma_ens(const __grid_constant__ EnsTab<float> tab, const CUtensorMap* __restrict__ maps, int in, int zero_arg) {
    using TT = TmaTile<BY, BZ>;
    extern __shared__ __align__(128) unsigned char sm[];
    pdl_wait();
    const int n = tab.n, total = tab.tbeg[n];
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(sm + ColTile<BY, BZ>::STAGE), 1);
        mbar_fence_init();
    }
    // the maps were written through the generic proxy (a host copy): acquire
    // them for the tensor-map proxy once per CTA, one map per thread
    for (int c = threadIdx.x; c < 4 * n; c += blockDim.x)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(maps + c) : "memory");
    __syncthreads();
    uint32_t phase = 0;
    int m = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        while (t >= tab.tbeg[m + 1]) ++m;          // items of a CTA increase, so m only advances
        const EnsMember<float>& M = tab.m[m];
        Scalars* sc = M.red.sc;
        if (*(volatile const int*)&sc->done) continue;
        const Dom& d = M.g.d;
        const int gx = (d.nx + TT::BX - 1) / TT::BX, gy = (d.ny + BY - 1) / BY;
        const int q = t - tab.tbeg[m];
        const int bx = q % gx, by = (q / gx) % gy, bz = q / (gx * gy);
        const bool zero_start = zero_arg == 1 || (zero_arg == 2 && sc->zflag);
        const CUtensorMap* mm = maps + 4 * m;
        if (!sor_col_block<BY, BZ, NT>(sm, mm + in, mm + 2, mm + 3, M.g, M.dl[in], M.rr, M.dl[1 - in], zero_start, sc,
                                       bx, by, bz, phase))
            return;
        phase ^= 1u;
        // the next block's copies overwrite the tiles: every thread is done with them
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
    }
}

// Persistent, double-buffered variant: each CTA walks tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ... and issues the copies of its next tile into the
// other shared-memory stage before computing the current one, so the copy
// latency hides behind compute.  cn1 and the per-plane coefficients come
// from a table over (plane, open-face mask) built once per handle with the
// same arithmetic as the scalar update.
template <int BY, int BZ>
struct PipeTile {
    using TT = TmaTile<BY, BZ>;
    static constexpr uint32_t STAGE = align_up(TT::OFF_CN, 128);          // d, r, f of one tile
    static constexpr uint32_t OFF_CN = 2 * STAGE;
    static constexpr uint32_t OFF_CT = OFF_CN + TT::RZ * 64 * 4;
    static constexpr uint32_t OFF_BAR = align_up(OFF_CT + 2 * TT::RZ * 4, 8);
    static constexpr uint32_t SMEM = OFF_BAR + 16;
};

template <int BY, int BZ, int NT>
__global__ void __launch_bounds__(NT)
k_sor_pipe(const __grid_constant__ CUtensorMap td, const __grid_constant__ CUtensorMap tr,
           const __grid_constant__ CUtensorMap tf, Geo<float> g, const float* __restrict__ cn1tab,
           float* __restrict__ dout, int zero_arg, Scalars* __restrict__ sc) {
    using TT = TmaTile<BY, BZ>;
    using PT = PipeTile<BY, BZ>;
    constexpr int BX = TT::BX, DXW = TT::DXW, FXW = TT::FXW, DY = TT::DY, DZ = TT::DZ, RY = TT::RY, RZ = TT::RZ;
    constexpr int NW = NT / 32;
    extern __shared__ __align__(128) unsigned char sm[];
    float(*sCN)[64] = reinterpret_cast<float(*)[64]>(sm + PT::OFF_CN);
    float* sCT = reinterpret_cast<float*>(sm + PT::OFF_CT);
    float* sCB = sCT + RZ;
    if (sc->done) return;
    const Dom& d = g.d;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = (d.nx + BX - 1) / BX, ty = (d.ny + BY - 1) / BY, tz = (d.nz + BZ - 1) / BZ;
    const int ntiles = tx * ty * tz;
    const bool zero_start = zero_arg == 1 || (zero_arg == 2 && sc->zflag);
    const uint32_t bar0 = smem_u32(sm + PT::OFF_BAR);
    auto origin = [&](int t, int& i0, int& j0, int& k0) {
        const int bx = t % tx, r_ = t / tx, by = r_ % ty, bz = r_ / ty;
        i0 = 1 + bx * BX;
        j0 = 1 + by * BY;
        k0 = 1 + bz * BZ;
    };
    auto issue = [&](int t, int st) {     // thread 0 only
        int i0, j0, k0;
        origin(t, i0, j0, k0);
        const int xd = i0 - 1, xf = xd & ~15;      // padded column of i0 - 4 (= 28 bx)
        unsigned char* base = sm + st * PT::STAGE;
        const uint32_t bar = bar0 + 8 * st;
        mbar_expect_tx(bar, TT::BYTES_R + TT::BYTES_F + (zero_start ? 0u : TT::BYTES_D));
        if (!zero_start) tma_load_3d(smem_u32(base), &td, xd, j0 - 2, k0 - 2, bar);
        tma_load_3d(smem_u32(base + TT::OFF_R), &tr, xd, j0 - 1, k0 - 1, bar);
        tma_load_3d(smem_u32(base + TT::OFF_F), &tf, xf, j0 - 1, k0 - 1, bar);
    };
    if (tid == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        mbar_fence_init();
        if (blockIdx.x < ntiles) issue(blockIdx.x, 0);
    }
    __syncthreads();
    uint32_t ph0 = 0u, ph1 = 0u;     // phase parity of each stage's barrier
    int st = 0;
    const float omega = g.omega, cx = g.cx, cy = g.cy;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int tn = t + gridDim.x;
        if (tid == 0 && tn < ntiles) issue(tn, st ^ 1);
        int i0, j0, k0;
        origin(t, i0, j0, k0);
        const int off = (i0 - 1) - ((i0 - 1) & ~15);  // flag tile offset, as in issue()
        float(*sD)[DY][DXW] = reinterpret_cast<float(*)[DY][DXW]>(sm + st * PT::STAGE);
        float(*sR)[RY][DXW] = reinterpret_cast<float(*)[RY][DXW]>(sm + st * PT::STAGE + TT::OFF_R);
        uint8_t(*sF)[RY][FXW] = reinterpret_cast<uint8_t(*)[RY][FXW]>(sm + st * PT::STAGE + TT::OFF_F);
        for (int q = tid; q < RZ * 64; q += NT) {
            const int kk = q >> 6, m = q & 63;
            const int k = min(max(k0 - 1 + kk, 0), d.nz + 1);
            sCN[kk][m] = cn1tab[k * 64 + m];
            if (m == 0) {
                sCT[kk] = g.cT[k];
                sCB[kk] = g.cB[k];
            }
        }
        if (zero_start) {
            float* p = &sD[0][0][0];
            for (int q = tid; q < DXW * DY * DZ; q += NT) p[q] = 0.f;
        }
        bool ok = false;
        const uint64_t t0 = global_ns();
        const uint32_t par = st ? ph1 : ph0;
        while (!(ok = mbar_try_wait(bar0 + 8 * st, par)))
            if (global_ns() - t0 > 1000000000ull) break;
        if (!__syncthreads_and(ok)) {
            if (tid == 0) atomicExch(&sc->timeout, 1);
            for (int s2 = 0; s2 < 2; ++s2) {          // bounded wait for copies still in flight
                const uint64_t t1 = global_ns();
                while (!mbar_try_wait(bar0 + 8 * s2, s2 ? ph1 : ph0))
                    if (global_ns() - t1 > 1000000000ull) break;
            }
            return;
        }
        if (st) ph1 ^= 1u;
        else ph0 ^= 1u;
        auto relax = [&](int x, int y, int z, int kz, uint8_t f, float rhs) {
            float ae = (f & F_E) ? cx : 0.f;
            float aw = (f & F_W) ? cx : 0.f;
            float an = (f & F_N) ? cy : 0.f;
            float as = (f & F_S) ? cy : 0.f;
            float at = (f & F_T) ? sCT[kz] : 0.f;
            float ab = (f & F_B) ? sCB[kz] : 0.f;
            const float cn1 = sCN[kz][f & 63];
            float s = 0.f;
            s += ae * sD[z][y][x + 1];
            s += aw * sD[z][y][x - 1];
            s += an * sD[z][y + 1][x];
            s += as * sD[z][y - 1][x];
            s += at * sD[z + 1][y][x];
            s += ab * sD[z - 1][y][x];
            float own = sD[z][y][x];
            float reltmp = omega * (cn1 * (s - rhs) - own);
            sD[z][y][x] = own + reltmp;
        };
        const int half = lane >> 4, m = lane & 15;
        for (int p = warp; 2 * p < RY * RZ; p += NW) {
            const int rw = 2 * p + half;
            if (rw < RY * RZ && m < (BX + 2) / 2) {
                const int jj = rw % RY, kk = rw / RY;
                const int ii = 2 * m + ((i0 + (j0 - 1 + jj) + (k0 - 1 + kk)) & 1);
                const uint8_t f = sF[kk][jj][ii + 3 + off];
                if (f & F_UNK) relax(ii + 3, jj + 1, kk + 1, kk, f, sR[kk][jj][ii + 3]);
            }
        }
        __syncthreads();
        for (int p = warp; 2 * p < BY * BZ; p += NW) {
            const int rw = 2 * p + half;
            if (rw < BY * BZ && m < BX / 2) {
                const int jj = rw % BY, kk = rw / BY;
                const int ii = 2 * m + ((i0 + (j0 + jj) + (k0 + kk)) & 1);
                const uint8_t f = sF[kk + 1][jj + 1][ii + 4 + off];
                if (f & F_UNK) relax(ii + 4, jj + 2, kk + 2, kk + 1, f, sR[kk + 1][jj + 1][ii + 4]);
            }
        }
        __syncthreads();
        const int i = i0 + lane;
        for (int rw = warp; rw < BY * BZ; rw += NW) {
            const int jj = rw % BY, kk = rw / BY;
            const int j = j0 + jj, k = k0 + kk;
            if (lane < BX && i <= d.nx && j <= d.ny && k <= d.nz && (sF[kk + 1][jj + 1][lane + 4 + off] & F_UNK))
                dout[(k * d.py + j) * d.px + i + OX] = sD[kk + 2][jj + 2][lane + 4];
        }
        __syncthreads();      // this stage is reloaded two tiles later
        st ^= 1;
    }
}

// k-marching variant: a CTA owns a 30 x TY column of cells over a chunk of
// planes [kb, ke) and walks it bottom to top with both colours in one pass
// (a wavefront two planes deep): red at plane k reads black neighbours at
// k-1 and k+1 that are still the old values (black k-1 is relaxed after red
// k), black at k-1 reads the new red values of k-2, k-1 (ring included) and
// k: the iterate of the in-order red-black sweep, bit for bit.  Each step
// takes two planes: red on planes 2t+1 and 2t+2 of the chunk (column plus a
// 1-cell ring), one barrier, then black on planes 2t and 2t+1 (column only)
// and their stores, whose cells are then final.  Red of the next step
// touches neither the cells black writes nor those it reads, so one barrier
// per step suffices.
//
// Each plane is one TMA copy of d (2-cell ring), r and the flags (1-cell
// ring) into one of NS shared-memory slots (plane q in slot q & (NS-1)) on
// its own mbarrier; the slots freed by a step are refilled right after its
// barrier, NS - 5 planes ahead of their first use, so the copies of later
// planes are in flight while the current ones are relaxed.  Only the x-y
// ring is loaded twice (by the neighbouring columns); planes are read once
// per chunk plus four halo planes.
//
// Lanes: 16 per row, two rows per warp (their colours differ, so the
// stride-2 shared-memory accesses of the two rows fall on opposite bank
// parities: no conflicts); a red row has 16 cells of the ring-extended
// 32-wide row, a black row 15 of the 30 interior cells, and the lane that
// relaxed the black cell of a pair stores the pair (8-byte aligned).  The
// update is branch-free: the four in-plane coefficients of an open-face
// mask come from a per-CTA table (one 16-byte read), the vertical ones and
// cn1 from the plane's slot.
//
// Periodic axes: the plane of a copy wraps on a periodic z axis; columns
// whose ring crosses a periodic x or y face overwrite the out-of-range rows
// and columns of each landed plane with plain loads of their images.
template <int TY, int NS>
struct MarchTile {
    static_assert((NS & (NS - 1)) == 0 && NS >= 8, "plane slots: a power of two, at least 8");
    static_assert(TY % 2 == 0, "rows come in pairs");
    static constexpr int TX = 30, W = 36, FW = 48;
    static constexpr int DY = TY + 4, RY = TY + 2;
    static constexpr int NW = RY / 2, NT = 32 * NW;       // one warp per red row pair
    static constexpr uint32_t BYTES_D = W * DY * 4;
    static constexpr uint32_t BYTES_R = W * RY * 4;
    static constexpr uint32_t BYTES_F = FW * RY;
    static constexpr uint32_t OFF_R = align_up(BYTES_D, 128);
    static constexpr uint32_t OFF_F = OFF_R + align_up(BYTES_R, 128);
    static constexpr uint32_t OFF_C = OFF_F + align_up(BYTES_F, 128);   // cn1 row [64], cT, cB
    static constexpr uint32_t SLOT = align_up(OFF_C + 66 * 4, 128);
    static constexpr uint32_t OFF_T4 = NS * SLOT;                         // float4 [64]: ae, aw, an, as
    static constexpr uint32_t OFF_BAR = OFF_T4 + 64 * 16;
    static constexpr uint32_t SMEM = OFF_BAR + NS * 8;
};

template <int TY, int NS>
__global__ void __launch_bounds__(MarchTile<TY, NS>::NT)
k_sor_march(const __grid_constant__ CUtensorMap td, const __grid_constant__ CUtensorMap tr,
            const __grid_constant__ CUtensorMap tf, Geo<float> g, const float* __restrict__ cn1tab,
            const float* __restrict__ din, const float* __restrict__ rin, float* __restrict__ dout, int kc,
            int zero_arg, Scalars* __restrict__ sc) {
    using MT = MarchTile<TY, NS>;
    constexpr int TX = MT::TX, W = MT::W, DY = MT::DY, RY = MT::RY, NT = MT::NT, NW = MT::NW;
    extern __shared__ __align__(128) unsigned char sm[];
    pdl_wait();
    if (sc->done) return;
    const Dom& d = g.d;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int half = lane >> 4, m = lane & 15;
    const int i0 = 1 + blockIdx.x * TX, j0 = 1 + blockIdx.y * TY;
    const int kb = 1 + blockIdx.z * kc, ke = min(kb + kc, d.nz + 1);
    const int nq = ke - kb + 4;                    // planes kb-2 .. ke+1 (slot index q = plane - kb + 2)
    const int xa = (i0 - 2 + OX) & ~3;             // padded column of the d and r boxes (16-byte aligned)
    const int xf = (i0 - 2 + OX) & ~15;            // of the flag box
    const int ox = OX - xa, oxf = OX - xf;         // shared column of cell i: i + ox (flags: i + oxf)
    const bool zero_start = zero_arg == 1 || (zero_arg == 2 && sc->zflag);
    const bool wrap_x = d.perx && (i0 - 2 < 1 || i0 + TX + 1 > d.nx);
    const bool wrap_y = d.pery && (j0 - 2 < 1 || j0 + TY + 1 > d.ny);
    const uint32_t bar0 = smem_u32(sm + MT::OFF_BAR);
    const float4* T4 = reinterpret_cast<const float4*>(sm + MT::OFF_T4);
    auto slot = [&](int q) { return sm + (uint32_t)(q & (NS - 1)) * MT::SLOT; };
    auto issue = [&](int q) {       // one thread
        const uint32_t bar = bar0 + 8u * (uint32_t)(q & (NS - 1));
        unsigned char* b = slot(q);
        int zc = kb - 2 + q;       // the plane the copy reads: the image on a periodic z axis
        if (d.perz && (zc < 1 || zc > d.nz)) zc = zc < 1 ? zc + d.nz : zc - d.nz;
        mbar_expect_tx(bar, MT::BYTES_R + MT::BYTES_F + (zero_start ? 0u : MT::BYTES_D));
        if (!zero_start) tma_load_3d(smem_u32(b), &td, xa, j0 - 2, zc, bar);
        tma_load_3d(smem_u32(b + MT::OFF_R), &tr, xa, j0 - 1, zc, bar);
        tma_load_3d(smem_u32(b + MT::OFF_F), &tf, xf, j0 - 1, zc, bar);
    };
    // coefficient row of slot q's plane (threads 0..65 of the group starting
    // at `first`) and, on a zero start, zeros for its d
    auto fill = [&](int q, int first) {
        const int e = tid - first;
        if (e >= 0 && e < 66) {
            const int k = coef_plane(d, kb - 2 + q);
            float* c = reinterpret_cast<float*>(slot(q) + MT::OFF_C);
            c[e] = e < 64 ? cn1tab[k * 64 + e] : (e == 64 ? g.cT[k] : g.cB[k]);
        }
        if (zero_start) {
            float* p = reinterpret_cast<float*>(slot(q));
            for (int x = tid; x < W * DY; x += NT) p[x] = 0.f;
        }
    };
    // images across a periodic x or y face of the ring cells of a landed plane
    auto fixup = [&](int q) {
        int k = kb - 2 + q;
        if (d.perz && (k < 1 || k > d.nz)) k = k < 1 ? k + d.nz : k - d.nz;
        unsigned char* b = slot(q);
        float* D = reinterpret_cast<float*>(b);
        float* R = reinterpret_cast<float*>(b + MT::OFF_R);
        uint8_t* F = b + MT::OFF_F;
        long long s_;
        for (int y = warp; y < DY; y += NW)
            for (int x = lane; x < TX + 4; x += 32) {
                const int i = i0 - 2 + x, j = j0 - 2 + y;
                const bool edge = (wrap_x && (i < 1 || i > d.nx)) || (wrap_y && (j < 1 || j > d.ny));
                if (!edge || !periodic_image(d, i, j, k, s_)) continue;
                if (!zero_start) D[y * W + i + ox] = s_ >= 0 ? din[s_] : 0.f;
                if (y >= 1 && y <= RY && x >= 1 && x <= TX + 2) {
                    R[(y - 1) * W + i + ox] = s_ >= 0 ? rin[s_] : 0.f;
                    F[(y - 1) * MT::FW + i + oxf] = s_ >= 0 ? g.flags[s_] : (uint8_t)0;
                }
            }
    };
    auto wait = [&](int q) {
        const uint32_t bar = bar0 + 8u * (uint32_t)(q & (NS - 1)), par = (uint32_t)(q / NS) & 1u;
        if (mbar_try_wait(bar, par)) return true;
        const uint64_t t0 = global_ns();
        while (!mbar_try_wait(bar, par))
            if (global_ns() - t0 > 1000000000ull) return false;
        return true;
    };
    const int nfirst = nq < NS ? nq : NS;
    if (tid == 0) {
        for (int q = 0; q < NS; ++q) mbar_init(bar0 + 8 * q, 1);
        mbar_fence_init();
        for (int q = 0; q < nfirst; ++q) issue(q);
    }
    for (int q = 0; q < nfirst; ++q) fill(q, 0);
    if (tid < 64) {
        const float cx = g.cx, cy = g.cy;
        reinterpret_cast<float4*>(sm + MT::OFF_T4)[tid] =
            make_float4((tid & F_E) ? cx : 0.f, (tid & F_W) ? cx : 0.f, (tid & F_N) ? cy : 0.f, (tid & F_S) ? cy : 0.f);
    }
    __syncthreads();
    int issued = nfirst, landed = 0;
    const float omega = g.omega;
    // the update of Sec. 2.6 at shared cell p of a plane whose slot starts at
    // S, with the same cell of the planes above (pt) and below (pb)
    auto relax = [&](const unsigned char* S, float* p, const float* pt, const float* pb, uint8_t f, float rhs) {
        const float* C = reinterpret_cast<const float*>(S + MT::OFF_C);
        const float4 a = T4[f & 63];
        const float cn1 = C[f & 63];
        const float at = (f & F_T) ? C[64] : 0.f, ab = (f & F_B) ? C[65] : 0.f;
        float s = 0.f;
        s += a.x * p[1];
        s += a.y * p[-1];
        s += a.z * p[W];
        s += a.w * p[-W];
        s += at * pt[0];
        s += ab * pb[0];
        float own = p[0];
        float reltmp = omega * (cn1 * (s - rhs) - own);
        p[0] = own + reltmp;
    };
    // this lane's cells: red row j0 - 1 + yr (16 cells from i0 - 1), black
    // row j0 + yr (15 cells from i0); shared offsets before the colour's
    // parity shift (floats from the slot base for d and r, bytes for flags)
    const int yr = 2 * warp + half;
    const int xr = i0 - 1 + 2 * m, xb = i0 + 2 * m;
    const int oDr = (yr + 1) * W + xr + ox, oRr = (int)(MT::OFF_R / 4) + yr * W + xr + ox;
    const int oFr = (int)MT::OFF_F + yr * MT::FW + xr + oxf;
    const int oDb = (yr + 2) * W + xb + ox, oRb = (int)(MT::OFF_R / 4) + (yr + 1) * W + xb + ox;
    const int oFb = (int)MT::OFF_F + (yr + 1) * MT::FW + xb + oxf;
    // parity of the first cell of this lane's red / black row on slot plane q: (pr0 + q) & 1
    const int pr0 = (i0 + (j0 - 1 + yr) + kb) & 1, pb0 = (i0 + (j0 + yr) + kb) & 1;
    const bool black_lane = warp < TY / 2 && m < TX / 2;
    const bool store_lane = black_lane && j0 + yr <= d.ny && xb <= d.nx;
    const bool store_pair = xb + 1 <= d.nx;
    float* const ob0 = dout + d.at(xb, j0 + yr, kb - 2);    // this lane's pair on slot plane 0
    const int nsteps = (nq - 1) / 2;
    for (int t = 0; t < nsteps; ++t) {
        // red planes 2t+1, 2t+2 read slots 2t .. 2t+3
        const int need = min(2 * t + 3, nq - 1);
        bool ok = true;
        while (landed <= need && ok) {
            ok = wait(landed);
            if (ok) ++landed;
        }
        if (wrap_x || wrap_y) {
            if (ok)
                for (int q = (t == 0 ? 0 : 2 * t + 2); q <= need; ++q) fixup(q);
            __syncthreads();
        }
        if (ok) {
#pragma unroll
            for (int h = 1; h <= 2; ++h) {
                const int q = 2 * t + h;
                if (q > nq - 2) break;
                unsigned char* S = slot(q);
                const int par = (pr0 + q) & 1;
                const uint8_t f = S[oFr + par];
                if (f & F_UNK) {
                    float* p = reinterpret_cast<float*>(S) + oDr + par;
                    relax(S, p, reinterpret_cast<const float*>(slot(q + 1)) + oDr + par,
                          reinterpret_cast<const float*>(slot(q - 1)) + oDr + par, f,
                          reinterpret_cast<const float*>(S)[oRr + par]);
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (!__syncthreads_and(ok)) {
            if (tid == 0) atomicExch(&sc->timeout, 1);
            for (int q = landed; q < issued; ++q) wait(q);      // bounded: copies still in flight land
            return;
        }
        // slots of planes 2t-3 and 2t-2 are free (their last readers, black
        // 2t-2 and 2t-1, finished before this barrier): planes up to 2t-2+NS
        const int lim = min(2 * t - 2 + NS, nq - 1);
        for (int g2 = 0; issued <= lim; ++g2, ++issued) {
            if (tid == 0) issue(issued);
            fill(issued, 66 * g2);
        }
        // black on planes 2t and 2t+1 (interior rows), then their stores
        if (black_lane) {
#pragma unroll
            for (int h = 0; h <= 1; ++h) {
                const int q = 2 * t + h;
                if (q < 2 || q > nq - 3) continue;
                unsigned char* S = slot(q);
                float* Sf = reinterpret_cast<float*>(S);
                const int par = (pb0 + q) & 1;
                const uint8_t f = S[oFb + par];
                if (f & F_UNK) {
                    float* p = Sf + oDb + par;
                    relax(S, p, reinterpret_cast<const float*>(slot(q + 1)) + oDb + par,
                          reinterpret_cast<const float*>(slot(q - 1)) + oDb + par, f, Sf[oRb + par]);
                }
                if (store_lane) {
                    float* o = ob0 + (long long)q * d.plane;
                    if (store_pair) {
                        *reinterpret_cast<float2*>(o) = make_float2(Sf[oDb], Sf[oDb + 1]);
                    } else {
                        *o = Sf[oDb];
                    }
                }
            }
        }
    }
}

template <int BY, int BZ, int NT>
cudaError_t allow_pipe() {
    return cudaFuncSetAttribute(k_sor_pipe<BY, BZ, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)PipeTile<BY, BZ>::SMEM);
}

template <int BY, int BZ, int NT>
int pipe_blocks() {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sor_pipe<BY, BZ, NT>, NT, PipeTile<BY, BZ>::SMEM);
    return sms * (per > 0 ? per : 1);
}

int g_pipe_blocks[4] = {0, 0, 0, 0};    // resident CTAs of each persistent config (set at prepare)

template <int BY, int BZ, int NT>
void launch_pipe_cfg(const Geo<float>& g, const TmaMaps& m, const float* cn1tab, int in, float* dout, int zero,
                     Scalars* sc, cudaStream_t s, int slot) {
    const Dom& d = g.d;
    const int blocks = g_pipe_blocks[slot] > 0 ? g_pipe_blocks[slot] : 152;
    const int ntiles = ((d.nx + 27) / 28) * ((d.ny + BY - 1) / BY) * ((d.nz + BZ - 1) / BZ);
    const int grid = ntiles < blocks ? ntiles : blocks;
    k_sor_pipe<BY, BZ, NT><<<grid, NT, PipeTile<BY, BZ>::SMEM, s>>>(m.d[in], m.r, m.f, g, cn1tab, dout, zero, sc);
}

template <int BY, int BZ, int NT>
cudaError_t allow_tma() {
    return cudaFuncSetAttribute(k_sor_tma<BY, BZ, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)TmaTile<BY, BZ>::SMEM);
}

template <int BY, int BZ, int NT>
void launch_tma_cfg(const Geo<float>& g, const TmaMaps& m, int in, float* dout, int zero, Scalars* sc,
                    cudaStream_t s) {
    const Dom& d = g.d;
    dim3 grid((d.nx + 27) / 28, (d.ny + BY - 1) / BY, (d.nz + BZ - 1) / BZ);
    launch_pdl(k_sor_tma<BY, BZ, NT>, grid, dim3(NT), TmaTile<BY, BZ>::SMEM, s, m.d[in], m.r, m.f, g, m.dptr[in],
               m.rptr, dout, zero, sc);
}

template <int BY, int BZ, int NT>
cudaError_t allow_col() {
    return cudaFuncSetAttribute(k_sor_col<BY, BZ, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ColTile<BY, BZ>::SMEM);
}

template <int BY, int BZ, int NT>
void launch_col_cfg(const Geo<float>& g, const TmaMaps& m, int in, float* dout, int zero, Scalars* sc,
                    cudaStream_t s, int pre) {
    const Dom& d = g.d;
    dim3 grid((d.nx + 27) / 28, (d.ny + BY - 1) / BY, (d.nz + BZ - 1) / BZ);
    launch_pdl(k_sor_col<BY, BZ, NT>, grid, dim3(NT), ColTile<BY, BZ>::SMEM, s, m.d[in], m.r, m.f, g, m.dptr[in],
               m.rptr, dout, zero, sc, pre);
}

template <int TY, int NS>
cudaError_t allow_march() {
    return cudaFuncSetAttribute(k_sor_march<TY, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)MarchTile<TY, NS>::SMEM);
}

int g_sms = 0;
int g_ens_tma_resident = 0;     // resident CTAs of the batched TMA ensemble sweep (set at prepare)

// planes per chunk: kc > 0 as given; kc <= 0: whole columns when they give at
// least two CTAs per SM, else the chunk length that does (at least 4 planes)
int march_chunk(const Dom& d, int ty, int kc) {
    if (kc > 0) return kc < d.nz ? kc : d.nz;
    const int cols = ((d.nx + 29) / 30) * ((d.ny + ty - 1) / ty);
    const int want = 2 * (g_sms > 0 ? g_sms : 152);
    const int chunks = (want + cols - 1) / cols;
    int c = (d.nz + chunks - 1) / chunks;
    if (c < 4) c = 4;
    return c < d.nz ? c : d.nz;
}

template <int TY, int NS>
void launch_march_cfg(const Geo<float>& g, const TmaMaps& m, const float* cn1tab, int in, float* dout, int kc,
                      int zero, Scalars* sc, cudaStream_t s) {
    const Dom& d = g.d;
    const int c = march_chunk(d, TY, kc);
    dim3 grid((d.nx + 29) / 30, (d.ny + TY - 1) / TY, (d.nz + c - 1) / c);
    launch_pdl(k_sor_march<TY, NS>, grid, dim3(MarchTile<TY, NS>::NT), MarchTile<TY, NS>::SMEM, s, m.d[in], m.r,
               m.f, g, cn1tab, m.dptr[in], m.rptr, dout, c, zero, sc);
}

using EncodeFn = PFN_cuTensorMapEncodeTiled_v12000;

EncodeFn encoder() {
    static EncodeFn fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeFn)p;
    }
    return fn;
}

bool encode3d(CUtensorMap* map, CUtensorMapDataType type, size_t es, void* base, const Dom& d, int bx, int by,
              int bz) {
    EncodeFn fn = encoder();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)d.px, (cuuint64_t)d.py, (cuuint64_t)(d.nz + 2)};
    cuuint64_t strides[2] = {(cuuint64_t)d.px * es, (cuuint64_t)d.px * d.py * es};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, type, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// (BY, BZ, threads) of the TMA tiles, in the order of their tile indices; the
// k-marching tiles (kFirstMarchCfg ..) as (TY, plane slots, threads)
const int kTmaCfg[kNumTmaTiles][3] = {{8, 8, 256}, {12, 12, 512}, {16, 12, 512}, {16, 16, 512},
                                      {8, 8, 256}, {8, 8, 512}, {16, 8, 512}, {12, 12, 512},
                                      {16, 16, 288}, {16, 8, 288}, {8, 16, 160}, {8, 8, 160},
                                      {8, 8, 256},   {8, 8, 320},   {8, 16, 320}, {16, 8, 512},
                                      {8, 8, 128},   {8, 8, 192}};

bool tma_supported(const Dom&) { return true; }

bool pipe_supported(const Dom& d) { return !d.perx && !d.pery && !d.perz; }

cudaError_t tma_prepare() {
    cudaError_t e = cudaSuccess, x;
    if ((x = allow_tma<8, 8, 256>()) != cudaSuccess) e = x;
    if ((x = allow_tma<12, 12, 512>()) != cudaSuccess) e = x;
    if ((x = allow_tma<16, 12, 512>()) != cudaSuccess) e = x;
    if ((x = allow_tma<16, 16, 512>()) != cudaSuccess) e = x;
    if ((x = allow_pipe<8, 8, 256>()) != cudaSuccess) e = x;
    if ((x = allow_pipe<8, 8, 512>()) != cudaSuccess) e = x;
    if ((x = allow_pipe<16, 8, 512>()) != cudaSuccess) e = x;
    if ((x = allow_pipe<12, 12, 512>()) != cudaSuccess) e = x;
    g_pipe_blocks[0] = pipe_blocks<8, 8, 256>();
    g_pipe_blocks[1] = pipe_blocks<8, 8, 512>();
    g_pipe_blocks[2] = pipe_blocks<16, 8, 512>();
    g_pipe_blocks[3] = pipe_blocks<12, 12, 512>();
    if ((x = allow_march<16, 16>()) != cudaSuccess) e = x;
    if ((x = allow_march<16, 8>()) != cudaSuccess) e = x;
    if ((x = allow_march<8, 16>()) != cudaSuccess) e = x;
    if ((x = allow_march<8, 8>()) != cudaSuccess) e = x;
    if ((x = allow_col<8, 8, 256>()) != cudaSuccess) e = x;
    if ((x = allow_col<8, 8, 320>()) != cudaSuccess) e = x;
    if ((x = allow_col<8, 16, 320>()) != cudaSuccess) e = x;
    if ((x = allow_col<16, 8, 512>()) != cudaSuccess) e = x;
    if ((x = allow_col<8, 8, 128>()) != cudaSuccess) e = x;
    if ((x = allow_col<8, 8, 192>()) != cudaSuccess) e = x;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if ((x = cudaFuncSetAttribute(k_sor_tma_ens<kEnsTmaBy, kEnsTmaBz, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)ColTile<kEnsTmaBy, kEnsTmaBz>::SMEM)) != cudaSuccess)
        e = x;
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sor_tma_ens<kEnsTmaBy, kEnsTmaBz, 256>, 256,
                                                  ColTile<kEnsTmaBy, kEnsTmaBz>::SMEM);
    g_ens_tma_resident = g_sms * (per > 0 ? per : 1);
    return e;
}

bool tma_encode(const Dom& d, float* dl0, float* dl1, float* rr, uint8_t* flags, TmaMaps* maps) {
    for (int c = 0; c < kNumTmaTiles; ++c) {
        const bool march = c >= kFirstMarchCfg && c < kFirstColCfg;
        const int by = kTmaCfg[c][0], bz = march ? -1 : kTmaCfg[c][1];    // march: one plane per copy
        TmaMaps& m = maps[c];
        m.dptr[0] = dl0;
        m.dptr[1] = dl1;
        m.rptr = rr;
        const int dz = march ? 1 : bz + 4;
        if (!encode3d(&m.d[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, dl0, d, 36, by + 4, dz)) return false;
        if (!encode3d(&m.d[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, dl1, d, 36, by + 4, dz)) return false;
        if (!encode3d(&m.r, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, rr, d, 36, by + 2, march ? 1 : bz + 2)) return false;
        if (!encode3d(&m.f, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, flags, d, 48, by + 2, march ? 1 : bz + 2)) return false;
    }
    return true;
}

int launch_sor_tma(const Geo<float>& g, const TmaMaps* maps, const float* cn1tab, int cfg, int kc, int in,
                   float* dout, int zero, Scalars* sc, cudaStream_t s, int pre) {
    const TmaMaps& m = maps[cfg];
    switch (cfg) {
        case 8: launch_march_cfg<16, 16>(g, m, cn1tab, in, dout, kc, zero, sc, s); break;
        case 9: launch_march_cfg<16, 8>(g, m, cn1tab, in, dout, kc, zero, sc, s); break;
        case 10: launch_march_cfg<8, 16>(g, m, cn1tab, in, dout, kc, zero, sc, s); break;
        case 11: launch_march_cfg<8, 8>(g, m, cn1tab, in, dout, kc, zero, sc, s); break;
        case 0: launch_tma_cfg<8, 8, 256>(g, m, in, dout, zero, sc, s); break;
        case 1: launch_tma_cfg<12, 12, 512>(g, m, in, dout, zero, sc, s); break;
        case 2: launch_tma_cfg<16, 12, 512>(g, m, in, dout, zero, sc, s); break;
        case 3: launch_tma_cfg<16, 16, 512>(g, m, in, dout, zero, sc, s); break;
        case 4: launch_pipe_cfg<8, 8, 256>(g, m, cn1tab, in, dout, zero, sc, s, 0); break;
        case 5: launch_pipe_cfg<8, 8, 512>(g, m, cn1tab, in, dout, zero, sc, s, 1); break;
        case 6: launch_pipe_cfg<16, 8, 512>(g, m, cn1tab, in, dout, zero, sc, s, 2); break;
        case 7: launch_pipe_cfg<12, 12, 512>(g, m, cn1tab, in, dout, zero, sc, s, 3); break;
        case 12: launch_col_cfg<8, 8, 256>(g, m, in, dout, zero, sc, s, pre); break;
        case 13: launch_col_cfg<8, 8, 320>(g, m, in, dout, zero, sc, s, pre); break;
        case 14: launch_col_cfg<8, 16, 320>(g, m, in, dout, zero, sc, s, pre); break;
        case 15: launch_col_cfg<16, 8, 512>(g, m, in, dout, zero, sc, s, pre); break;
        case 16: launch_col_cfg<8, 8, 128>(g, m, in, dout, zero, sc, s, pre); break;
        case 17: launch_col_cfg<8, 8, 192>(g, m, in, dout, zero, sc, s, pre); break;
        default: break;
    }
    return 1;
}

bool tma_encode_member(const Dom& d, float* dl0, float* dl1, float* rr, const uint8_t* flags, CUtensorMap* out4) {
    constexpr int by = kEnsTmaBy, bz = kEnsTmaBz;
    return encode3d(&out4[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, dl0, d, 36, by + 4, bz + 4) &&
           encode3d(&out4[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, dl1, d, 36, by + 4, bz + 4) &&
           encode3d(&out4[2], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, rr, d, 36, by + 2, bz + 2) &&
           encode3d(&out4[3], CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, const_cast<uint8_t*>(flags), d, 48, by + 2, bz + 2);
}

// tensor maps of the TMA estimate (32 x 8 x 8 cells per CTA): d[0], d[1] with a
// 1-cell ring in a 40-wide box (x from the padded column of i0 - 4), r (the
// block, x from the padded column of i0) and the flags (48 wide from the
// 16-byte column at or below that of i0 - 4)
bool tma_encode_est(const Dom& d, float* dl0, float* dl1, float* rr, const uint8_t* flags, CUtensorMap* out4) {
    return encode3d(&out4[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, dl0, d, 40, 10, 10) &&
           encode3d(&out4[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, dl1, d, 40, 10, 10) &&
           encode3d(&out4[2], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, rr, d, 32, 8, 8) &&
           encode3d(&out4[3], CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, const_cast<uint8_t*>(flags), d, 48, 8, 8);
}

int sor_tma_ens_resident() { return g_ens_tma_resident; }

int launch_sor_tma_ens(const EnsTab<float>& tab, const CUtensorMap* maps, int in, int zero, int ctas,
                       cudaStream_t s) {
    const int total = tab.tbeg[tab.n];
    const int grid = ctas < total ? ctas : total;
    if (grid < 1) return 0;
    launch_pdl(k_sor_tma_ens<kEnsTmaBy, kEnsTmaBz, 256>, dim3(grid), dim3(256), ColTile<kEnsTmaBy, kEnsTmaBz>::SMEM,
               s, tab, maps, in, zero);
    return 1;
}

// cn1 over (plane, open-face mask): the same sum and division as the update
__global__ void k_cn1_table(Geo<float> g, float* tab) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (g.d.nz + 2) * 64) return;
    const int k = q >> 6, m = q & 63;
    float ae = (m & F_E) ? g.cx : 0.f;
    float aw = (m & F_W) ? g.cx : 0.f;
    float an = (m & F_N) ? g.cy : 0.f;
    float as = (m & F_S) ? g.cy : 0.f;
    float at = (m & F_T) ? g.cT[k] : 0.f;
    float ab = (m & F_B) ? g.cB[k] : 0.f;
    const float sum = ae + aw + an + as + at + ab;
    tab[q] = sum > 0.f ? 1.f / sum : 0.f;
}

// rows of the column-walk sweeps' coefficient table (les_tma.cuh, kColRow)
__global__ void k_col_table(Geo<float> g, const float* cn1tab, float* tab) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int rows = g.d.nz + 2 + kColTableRows;
    if (q >= rows * kColRow) return;
    const int r = q / kColRow, e = q % kColRow;
    const int k = coef_plane(g.d, r);
    tab[q] = e < 64 ? cn1tab[k * 64 + e] : (e == 64 ? g.cT[k] : (e == 65 ? g.cB[k] : 0.f));
}

int launch_col_table(const Geo<float>& g, const float* cn1tab, float* tab, cudaStream_t s) {
    const int n = (g.d.nz + 2 + kColTableRows) * kColRow;
    k_col_table<<<(n + 255) / 256, 256, 0, s>>>(g, cn1tab, tab);
    return 1;
}

int launch_cn1_table(const Geo<float>& g, float* tab, cudaStream_t s) {
    const int n = (g.d.nz + 2) * 64;
    k_cn1_table<<<(n + 255) / 256, 256, 0, s>>>(g, tab);
    return 1;
}

// Self-test of the bounded device wait used by the TMA sweeps: an mbarrier
// armed for 16 bytes of transaction that no copy will ever deliver.  The wait
// gives up after limit_ns (global timer), every thread agrees, and the block
// reports the timeout and returns; nothing is in flight, so the context stays
// usable.  status: 1 = timed out (expected), 0 = the barrier completed.
__global__ void k_wait_selftest(unsigned long long limit_ns, int* status) {
    __shared__ __align__(8) uint64_t bar_word;
    const uint32_t bar = smem_u32(&bar_word);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_expect_tx(bar, 16);
    __syncthreads();
    bool ok = false;
    const uint64_t t0 = global_ns();
    while (!(ok = mbar_try_wait(bar, 0)))
        if (global_ns() - t0 > limit_ns) break;
    const bool all = __syncthreads_and(ok);
    if (threadIdx.x == 0) {
        *status = all ? 0 : 1;
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
    }
}

int launch_wait_selftest(unsigned long long limit_ns, int* status, cudaStream_t s) {
    k_wait_selftest<<<1, 128, 0, s>>>(limit_ns, status);
    return 1;
}

}  // namespace les
