// Fused red-black SOR sweep (Sec. 2.6): one launch performs the red and the
// black half-sweep of the correction equation A d = r, reading d_in and
// writing d_out (ping-pong), so the result is exactly the in-place two-pass
// red-black sweep.
//
// Each CTA owns a TX x TY column tile of one k-chunk and marches up in k
// keeping four d planes (tile + 2-cell halo) in shared memory:
//   step kc: load d_in plane kc+1 and r/flags plane kc,
//            red cells of plane kc on tile+1 (needs black-old at kc-1..kc+1),
//            black cells of plane kc-1 on the tile (needs red-new at kc-2..kc),
//            store plane kc-1 of the tile.
// Red values on the 1-cell ring are recomputed redundantly from the same
// black-old inputs as in the neighbouring CTA, so every CTA sees the same red
// iterate and no inter-CTA synchronisation is needed.  The halo re-reads hit
// L2; DRAM traffic per sweep is ~ d in, r in, flags in, d out = 13 B/cell.
#include <type_traits>

#include "les_internal.cuh"

namespace les {

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX / 2 * TY)
k_sor_fused(Geo<T> g, const T* __restrict__ din, T* __restrict__ dout, const T* __restrict__ r,
            int zero_arg, const Scalars* __restrict__ sc, int kc_len) {
    constexpr int NT = TX / 2 * TY;
    constexpr int DX = TX + 4, DY = TY + 4;
    constexpr int RX = TX + 2, RY = TY + 2;
    __shared__ T sD[4][DY][DX];
    __shared__ T sR[2][RY][RX];
    __shared__ uint8_t sF[2][RY][RX];

    const Dom& d = g.d;
    const int tid = threadIdx.x;
    const int i0 = 1 + blockIdx.x * TX;
    const int j0 = 1 + blockIdx.y * TY;
    const int k0 = 1 + blockIdx.z * kc_len;
    const int k1 = min(k0 + kc_len, d.nz + 1);   // chunk is [k0, k1)
    const T omega = g.omega;
    if (sc->done) return;
    const bool zero_start = zero_arg == 1 || (zero_arg == 2 && sc->zflag);

    // padded index of (i, j, k) with periodic wrap; false outside the padded box
    auto src = [&](int i, int j, int k, long long& q) -> bool {
        if (d.perx) { i = i < 1 ? i + d.nx : (i > d.nx ? i - d.nx : i); }
        else if (i < 0 || i > d.nx + 1) return false;
        if (d.pery) { j = j < 1 ? j + d.ny : (j > d.ny ? j - d.ny : j); }
        else if (j < 0 || j > d.ny + 1) return false;
        if (d.perz) { k = k < 1 ? k + d.nz : (k > d.nz ? k - d.nz : k); }
        else if (k < 0 || k > d.nz + 1) return false;
        q = d.at(i, j, k);
        return true;
    };
    auto load_d = [&](int kk) {
        T(*P)[DX] = sD[kk & 3];
        for (int q = tid; q < DX * DY; q += NT) {
            const int ii = q % DX, jj = q / DX;
            long long s;
            T v = T(0);
            if (!zero_start && src(i0 - 2 + ii, j0 - 2 + jj, kk, s)) v = din[s];
            P[jj][ii] = v;
        }
    };
    auto load_rf = [&](int kk) {
        T(*R)[RX] = sR[kk & 1];
        uint8_t(*F)[RX] = sF[kk & 1];
        for (int q = tid; q < RX * RY; q += NT) {
            const int ii = q % RX, jj = q / RX;
            long long s;
            T rv = T(0);
            uint8_t fv = 0;
            if (src(i0 - 1 + ii, j0 - 1 + jj, kk, s)) {
                fv = g.flags[s];
                if (fv & F_UNK) rv = r[s];
            }
            R[jj][ii] = rv;
            F[jj][ii] = fv;
        }
    };
    // the printed update, at shared-memory position (x, y) of plane kk
    auto relax = [&](int kk, int x, int y, uint8_t f, T rhs) {
        T ae = (f & F_E) ? g.cx : T(0);
        T aw = (f & F_W) ? g.cx : T(0);
        T an = (f & F_N) ? g.cy : T(0);
        T as = (f & F_S) ? g.cy : T(0);
        const int kz = min(max(kk, 0), d.nz + 1);
        const int kl = d.perz ? (kk < 1 ? kk + d.nz : (kk > d.nz ? kk - d.nz : kk)) : kz;
        T at = (f & F_T) ? g.cT[kl] : T(0);
        T ab = (f & F_B) ? g.cB[kl] : T(0);
        T cn1 = T(1) / (ae + aw + an + as + at + ab);
        const T(*P)[DX] = sD[kk & 3];
        T s = T(0);
        s += ae * P[y][x + 1];
        s += aw * P[y][x - 1];
        s += an * P[y + 1][x];
        s += as * P[y - 1][x];
        s += at * sD[(kk + 1) & 3][y][x];
        s += ab * sD[(kk - 1) & 3][y][x];
        T own = P[y][x];
        T reltmp = omega * (cn1 * (s - rhs) - own);
        sD[kk & 3][y][x] = own + reltmp;
    };

    load_d(k0 - 2);
    load_d(k0 - 1);
    for (int kc = k0 - 1; kc <= k1; ++kc) {
        load_d(kc + 1);
        load_rf(kc);
        __syncthreads();
        // red (i+j+k odd) on plane kc, tile + 1-cell ring
        for (int q = tid; q < (RX / 2) * RY; q += NT) {
            const int jj = q / (RX / 2), m = q % (RX / 2);
            const int par = (i0 + (j0 - 1 + jj) + kc) & 1;
            const int ii = 2 * m + par;
            const uint8_t f = sF[kc & 1][jj][ii];
            if (f & F_UNK) relax(kc, ii + 1, jj + 1, f, sR[kc & 1][jj][ii]);
        }
        __syncthreads();
        const int kb = kc - 1;
        if (kb >= k0) {
            // black (i+j+k even) on plane kb, tile only
            for (int q = tid; q < (TX / 2) * TY; q += NT) {
                const int jj = q / (TX / 2), m = q % (TX / 2);
                const int par = (i0 + (j0 + jj) + kb) & 1;
                const int ii = 2 * m + par;
                const uint8_t f = sF[kb & 1][jj + 1][ii + 1];
                if (f & F_UNK) relax(kb, ii + 2, jj + 2, f, sR[kb & 1][jj + 1][ii + 1]);
            }
            __syncthreads();
            for (int q = tid; q < TX * TY; q += NT) {
                const int ii = q % TX, jj = q / TX;
                const int i = i0 + ii, j = j0 + jj;
                if (i <= d.nx && j <= d.ny && (sF[kb & 1][jj + 1][ii + 1] & F_UNK))
                    dout[d.at(i, j, kb)] = sD[kb & 3][jj + 2][ii + 2];
            }
        }
        __syncthreads();
    }
}

// 3-D block variant for grids that fit in L2: no marching, so thousands of
// independent CTAs hide the load latency.  One CTA loads d on its BX x BY x BZ
// block plus a 2-cell halo and r/flags on block + 1, updates the red cells of
// block + 1 ring, then the black cells of the block, and stores the block.
template <typename T, int BX, int BY, int BZ>
__global__ void __launch_bounds__(256)
k_sor_block(Geo<T> g, const T* __restrict__ din, T* __restrict__ dout, const T* __restrict__ r, int zero_arg,
            const Scalars* __restrict__ sc) {
    constexpr int NT = 256;
    constexpr int DX = BX + 4, DY = BY + 4, DZ = BZ + 4;
    constexpr int RX = BX + 2, RY = BY + 2, RZ = BZ + 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T(*sD)[DY][DX] = reinterpret_cast<T(*)[DY][DX]>(smem_raw);
    T(*sR)[RY][RX] = reinterpret_cast<T(*)[RY][RX]>(smem_raw + sizeof(T) * DX * DY * DZ);
    uint8_t(*sF)[RY][RX] = reinterpret_cast<uint8_t(*)[RY][RX]>(smem_raw + sizeof(T) * (DX * DY * DZ + RX * RY * RZ));
    const Dom& d = g.d;
    const int tid = threadIdx.x;
    const int i0 = 1 + blockIdx.x * BX, j0 = 1 + blockIdx.y * BY, k0 = 1 + blockIdx.z * BZ;
    const T omega = g.omega;
    if (sc->done) return;
    const bool zero_start = zero_arg == 1 || (zero_arg == 2 && sc->zflag);
    auto src = [&](int i, int j, int k, long long& q) -> bool {
        if (d.perx) { i = i < 1 ? i + d.nx : (i > d.nx ? i - d.nx : i); }
        else if (i < 0 || i > d.nx + 1) return false;
        if (d.pery) { j = j < 1 ? j + d.ny : (j > d.ny ? j - d.ny : j); }
        else if (j < 0 || j > d.ny + 1) return false;
        if (d.perz) { k = k < 1 ? k + d.nz : (k > d.nz ? k - d.nz : k); }
        else if (k < 0 || k > d.nz + 1) return false;
        q = d.at(i, j, k);
        return true;
    };
    // Every thread stages its share of the three tiles in registers first, so
    // all of its loads are in flight together; blocks whose halo lies inside
    // the padded box and needs no periodic wrap use plain address arithmetic.
    constexpr int ND = DX * DY * DZ, NR = RX * RY * RZ;
    constexpr int LD = (ND + NT - 1) / NT, LR = (NR + NT - 1) / NT;
    // (halo strictly inside 1..n: periodic ghosts of d are never maintained)
    const bool inner = i0 - 2 >= 1 && i0 + BX + 1 <= d.nx && j0 - 2 >= 1 && j0 + BY + 1 <= d.ny &&
                       k0 - 2 >= 1 && k0 + BZ + 1 <= d.nz;
    T* sDf = &sD[0][0][0];
    T* sRf = &sR[0][0][0];
    uint8_t* sFf = &sF[0][0][0];
    const long long bd = d.at(i0 - 2, j0 - 2, k0 - 2);
    const long long br = d.at(i0 - 1, j0 - 1, k0 - 1);
    T vd[LD];
    T vr[LR];
    uint8_t vf[LR];
#pragma unroll
    for (int n = 0; n < LD; ++n) {
        const int q = tid + n * NT;
        vd[n] = T(0);
        if (q < ND && !zero_start) {
            const int ii = q % DX, t = q / DX, jj = t % DY, kk = t / DY;
            long long a = bd + ((long long)kk * d.py + jj) * d.px + ii;
            bool ok = true;
            if (!inner) ok = src(i0 - 2 + ii, j0 - 2 + jj, k0 - 2 + kk, a);
            if (ok) vd[n] = din[a];
        }
    }
#pragma unroll
    for (int n = 0; n < LR; ++n) {
        const int q = tid + n * NT;
        vf[n] = 0;
        vr[n] = T(0);
        if (q < NR) {
            const int ii = q % RX, t = q / RX, jj = t % RY, kk = t / RY;
            long long a = br + ((long long)kk * d.py + jj) * d.px + ii;
            bool ok = true;
            if (!inner) ok = src(i0 - 1 + ii, j0 - 1 + jj, k0 - 1 + kk, a);
            if (ok) {
                vf[n] = g.flags[a];
                vr[n] = r[a];
            }
        }
    }
#pragma unroll
    for (int n = 0; n < LD; ++n) {
        const int q = tid + n * NT;
        if (q < ND) sDf[q] = vd[n];
    }
#pragma unroll
    for (int n = 0; n < LR; ++n) {
        const int q = tid + n * NT;
        if (q < NR) {
            sRf[q] = (vf[n] & F_UNK) ? vr[n] : T(0);
            sFf[q] = vf[n];
        }
    }
    __syncthreads();
    // the printed update at shared position (x, y, z) of the d tile
    auto relax = [&](int x, int y, int z, int kglob, uint8_t f, T rhs) {
        T ae = (f & F_E) ? g.cx : T(0);
        T aw = (f & F_W) ? g.cx : T(0);
        T an = (f & F_N) ? g.cy : T(0);
        T as = (f & F_S) ? g.cy : T(0);
        const int kl = d.perz ? (kglob < 1 ? kglob + d.nz : (kglob > d.nz ? kglob - d.nz : kglob))
                              : min(max(kglob, 0), d.nz + 1);
        T at = (f & F_T) ? g.cT[kl] : T(0);
        T ab = (f & F_B) ? g.cB[kl] : T(0);
        T cn1 = T(1) / (ae + aw + an + as + at + ab);
        T s = T(0);
        s += ae * sD[z][y][x + 1];
        s += aw * sD[z][y][x - 1];
        s += an * sD[z][y + 1][x];
        s += as * sD[z][y - 1][x];
        s += at * sD[z + 1][y][x];
        s += ab * sD[z - 1][y][x];
        T own = sD[z][y][x];
        T reltmp = omega * (cn1 * (s - rhs) - own);
        sD[z][y][x] = own + reltmp;
    };
    // red (i+j+k odd) on block + 1 ring
    for (int q = tid; q < (RX / 2) * RY * RZ; q += NT) {
        const int m = q % (RX / 2), t = q / (RX / 2), jj = t % RY, kk = t / RY;
        const int par = (i0 + (j0 - 1 + jj) + (k0 - 1 + kk)) & 1;
        const int ii = 2 * m + par;
        const uint8_t f = sF[kk][jj][ii];
        if (f & F_UNK) relax(ii + 1, jj + 1, kk + 1, k0 - 1 + kk, f, sR[kk][jj][ii]);
    }
    __syncthreads();
    // black (i+j+k even) on the block
    for (int q = tid; q < (BX / 2) * BY * BZ; q += NT) {
        const int m = q % (BX / 2), t = q / (BX / 2), jj = t % BY, kk = t / BY;
        const int par = (i0 + (j0 + jj) + (k0 + kk)) & 1;
        const int ii = 2 * m + par;
        const uint8_t f = sF[kk + 1][jj + 1][ii + 1];
        if (f & F_UNK) relax(ii + 2, jj + 2, kk + 2, k0 + kk, f, sR[kk + 1][jj + 1][ii + 1]);
    }
    __syncthreads();
    for (int q = tid; q < BX * BY * BZ; q += NT) {
        const int ii = q % BX, t = q / BX, jj = t % BY, kk = t / BY;
        const int i = i0 + ii, j = j0 + jj, k = k0 + kk;
        if (i <= d.nx && j <= d.ny && k <= d.nz && (sF[kk + 1][jj + 1][ii + 1] & F_UNK))
            dout[d.at(i, j, k)] = sD[kk + 2][jj + 2][ii + 2];
    }
}

// Row-mapped 3-D block variant (28 x BY x BZ): the d tile is 32 cells wide,
// so each halo row is one warp-wide coalesced load; per-lane column offsets
// and per-row offsets are computed once (32-bit), and cn1 comes from a
// per-CTA table over (plane, open-face mask) built with the same arithmetic
// as the scalar update, so the iterate is bit-identical to the other kernels.
template <typename T, int BY, int BZ>
struct RowTile {
    static constexpr int BX = 28, DX = 32, DY = BY + 4, DZ = BZ + 4, RY = BY + 2, RZ = BZ + 2;
    static constexpr size_t smem() {
        return sizeof(T) * (DZ * DY * DX + RZ * RY * 32 + RZ * 64 + 2 * RZ) + RZ * RY * 32;
    }
};

// one 28 x BY x BZ tile (bx, by, bz) of the sweep; the caller has checked `done`
template <typename T, int BY, int BZ>
__device__ __forceinline__ void sor_rows_tile(const Geo<T>& g, const T* __restrict__ din, T* __restrict__ dout,
                                              const T* __restrict__ r, bool zero_start, int bx, int by, int bz,
                                              unsigned char* smem_raw) {
    using RT = RowTile<T, BY, BZ>;
    constexpr int DX = RT::DX, DY = RT::DY, DZ = RT::DZ, RY = RT::RY, RZ = RT::RZ, BX = RT::BX;
    T(*sD)[DY][DX] = reinterpret_cast<T(*)[DY][DX]>(smem_raw);
    T(*sR)[RY][32] = reinterpret_cast<T(*)[RY][32]>(smem_raw + sizeof(T) * DZ * DY * DX);
    T(*sCN)[64] = reinterpret_cast<T(*)[64]>(smem_raw + sizeof(T) * (DZ * DY * DX + RZ * RY * 32));
    T* sCT = reinterpret_cast<T*>(smem_raw + sizeof(T) * (DZ * DY * DX + RZ * RY * 32 + RZ * 64));
    T* sCB = sCT + RZ;
    uint8_t(*sF)[RY][32] =
        reinterpret_cast<uint8_t(*)[RY][32]>(smem_raw + sizeof(T) * (DZ * DY * DX + RZ * RY * 32 + RZ * 64 + 2 * RZ));
    const Dom& d = g.d;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int i0 = 1 + bx * BX, j0 = 1 + by * BY, k0 = 1 + bz * BZ;
    const int px = d.px, py = d.py;
    // column offset of a lane (wrapped on a periodic axis), -1 outside the padded box
    auto col = [&](int i) -> int {
        if (d.perx) i = i < 1 ? i + d.nx : (i > d.nx ? i - d.nx : i);
        else if (i < 0 || i > d.nx + 1) return -1;
        return i + OX;
    };
    auto row = [&](int j, int k) -> int {
        if (d.pery) j = j < 1 ? j + d.ny : (j > d.ny ? j - d.ny : j);
        else if (j < 0 || j > d.ny + 1) return -1;
        if (d.perz) k = k < 1 ? k + d.nz : (k > d.nz ? k - d.nz : k);
        else if (k < 0 || k > d.nz + 1) return -1;
        return (k * py + j) * px;
    };
    const int cD = col(i0 - 2 + lane);
    const int cR = lane < BX + 2 ? col(i0 - 1 + lane) : -1;
    constexpr int ND = (DY * DZ + 7) / 8, NR = (RY * RZ + 7) / 8;
    T vd[ND];
    T vr[NR];
    uint8_t vf[NR];
#pragma unroll
    for (int n = 0; n < ND; ++n) {
        const int rw = warp + 8 * n;
        vd[n] = T(0);
        if (rw < DY * DZ && !zero_start) {
            const int ro = row(j0 - 2 + rw % DY, k0 - 2 + rw / DY);
            if (ro >= 0 && cD >= 0) vd[n] = din[ro + cD];
        }
    }
#pragma unroll
    for (int n = 0; n < NR; ++n) {
        const int rw = warp + 8 * n;
        vf[n] = 0;
        vr[n] = T(0);
        if (rw < RY * RZ) {
            const int ro = row(j0 - 1 + rw % RY, k0 - 1 + rw / RY);
            if (ro >= 0 && cR >= 0) {
                vf[n] = g.flags[ro + cR];
                vr[n] = r[ro + cR];
            }
        }
    }
    // per-plane coefficients and the cn1 table over the six open-face bits
    // (from the handle's table on FP32 grids, else the same arithmetic here)
    for (int q = tid; q < RZ * 64; q += 256) {
        const int kk = q >> 6, m = q & 63;
        int k = k0 - 1 + kk;
        k = d.perz ? (k < 1 ? k + d.nz : (k > d.nz ? k - d.nz : k)) : min(max(k, 0), d.nz + 1);
        const T ct = g.cT[k], cb = g.cB[k];
        if (g.cn1) {
            sCN[kk][m] = g.cn1[k * 64 + m];
        } else {
            T ae = (m & F_E) ? g.cx : T(0);
            T aw = (m & F_W) ? g.cx : T(0);
            T an = (m & F_N) ? g.cy : T(0);
            T as = (m & F_S) ? g.cy : T(0);
            T at = (m & F_T) ? ct : T(0);
            T ab = (m & F_B) ? cb : T(0);
            const T sum = ae + aw + an + as + at + ab;
            sCN[kk][m] = sum > T(0) ? T(1) / sum : T(0);
        }
        if (m == 0) {
            sCT[kk] = ct;
            sCB[kk] = cb;
        }
    }
#pragma unroll
    for (int n = 0; n < ND; ++n) {
        const int rw = warp + 8 * n;
        if (rw < DY * DZ) sD[rw / DY][rw % DY][lane] = vd[n];
    }
#pragma unroll
    for (int n = 0; n < NR; ++n) {
        const int rw = warp + 8 * n;
        if (rw < RY * RZ) {
            sR[rw / RY][rw % RY][lane] = (vf[n] & F_UNK) ? vr[n] : T(0);
            sF[rw / RY][rw % RY][lane] = vf[n];
        }
    }
    __syncthreads();
    const T omega = g.omega, cx = g.cx, cy = g.cy;
    auto relax = [&](int x, int y, int z, int kz, uint8_t f, T rhs) {
        const T ct = sCT[kz], cb = sCB[kz];
        const T cn1 = sCN[kz][f & 63];
        T s = T(0);
        if ((f & 63) == 63) {
            // all six faces open: the same sum without the selects
            s += cx * sD[z][y][x + 1];
            s += cx * sD[z][y][x - 1];
            s += cy * sD[z][y + 1][x];
            s += cy * sD[z][y - 1][x];
            s += ct * sD[z + 1][y][x];
            s += cb * sD[z - 1][y][x];
        } else {
            const T ae = (f & F_E) ? cx : T(0), aw = (f & F_W) ? cx : T(0);
            const T an = (f & F_N) ? cy : T(0), as = (f & F_S) ? cy : T(0);
            const T at = (f & F_T) ? ct : T(0), ab = (f & F_B) ? cb : T(0);
            s += ae * sD[z][y][x + 1];
            s += aw * sD[z][y][x - 1];
            s += an * sD[z][y + 1][x];
            s += as * sD[z][y - 1][x];
            s += at * sD[z + 1][y][x];
            s += ab * sD[z - 1][y][x];
        }
        T own = sD[z][y][x];
        T reltmp = omega * (cn1 * (s - rhs) - own);
        sD[z][y][x] = own + reltmp;
    };
    // red (i+j+k odd) on block + 1 ring: 15 per 30-wide row, two rows per warp pass
    const int half = lane >> 4, m = lane & 15;
    for (int p = warp; 2 * p < RY * RZ; p += 8) {
        const int rw = 2 * p + half;
        if (rw < RY * RZ && m < (BX + 2) / 2) {
            const int jj = rw % RY, kk = rw / RY;
            const int ii = 2 * m + ((i0 + (j0 - 1 + jj) + (k0 - 1 + kk)) & 1);
            const uint8_t f = sF[kk][jj][ii];
            if (f & F_UNK) relax(ii + 1, jj + 1, kk + 1, kk, f, sR[kk][jj][ii]);
        }
    }
    __syncthreads();
    // black (i+j+k even) on the block: 14 per row
    for (int p = warp; 2 * p < BY * BZ; p += 8) {
        const int rw = 2 * p + half;
        if (rw < BY * BZ && m < BX / 2) {
            const int jj = rw % BY, kk = rw / BY;
            const int ii = 2 * m + ((i0 + (j0 + jj) + (k0 + kk)) & 1);
            const uint8_t f = sF[kk + 1][jj + 1][ii + 1];
            if (f & F_UNK) relax(ii + 2, jj + 2, kk + 2, kk + 1, f, sR[kk + 1][jj + 1][ii + 1]);
        }
    }
    __syncthreads();
    // store the block (cells that are not unknowns hold 0 in d and in the tile)
    const int i = i0 + lane;
    if (lane < BX && i <= d.nx) {
        const int kend = min(BZ, d.nz + 1 - k0), jend = min(BY, d.ny + 1 - j0);
        for (int rw = warp; rw < BY * BZ; rw += 8) {
            const int jj = rw % BY, kk = rw / BY;
            if (jj < jend && kk < kend) dout[((k0 + kk) * py + j0 + jj) * px + i + OX] = sD[kk + 2][jj + 2][lane + 2];
        }
    }
}

template <typename T, int BY, int BZ>
__global__ void __launch_bounds__(256)
k_sor_rows(Geo<T> g, const T* __restrict__ din, T* __restrict__ dout, const T* __restrict__ r, int zero_arg,
           const Scalars* __restrict__ sc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (sc->done) return;
    const bool zero_start = zero_arg == 1 || (zero_arg == 2 && sc->zflag);
    sor_rows_tile<T, BY, BZ>(g, din, dout, r, zero_start, blockIdx.x, blockIdx.y, blockIdx.z, smem_raw);
}

// The ensemble sweep: one persistent launch over the tiles of every member
// (flattened in member order); each CTA walks its share of the list, skips
// the tiles of members whose solve is done, and relaxes the others with the
// same tile code as the single-domain launch (bit-identical iterates).
template <typename T, int BY, int BZ>
__global__ void __launch_bounds__(256) k_sor_rows_ens(const __grid_constant__ EnsTab<T> tab, int in, int zero_arg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int total = tab.sbeg[tab.n];
    int m = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        while (t >= tab.sbeg[m + 1]) ++m;
        const EnsMember<T>& M = tab.m[m];
        if (M.red.sc->done) continue;                     // uniform over the CTA
        const bool zero_start = zero_arg == 1 || (zero_arg == 2 && M.red.sc->zflag);
        const int lt = t - tab.sbeg[m], sx = M.sgrid[0], sy = M.sgrid[1];
        sor_rows_tile<T, BY, BZ>(M.g, M.dl[in], M.dl[1 - in], M.rr, zero_start, lt % sx, (lt / sx) % sy,
                                 lt / (sx * sy), smem_raw);
        __syncthreads();                                  // shared tiles are reused by the next item
    }
}

template <typename T, int BY, int BZ>
static cudaError_t allow_rows() {
    cudaError_t e = cudaFuncSetAttribute(k_sor_rows<T, BY, BZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)RowTile<T, BY, BZ>::smem());
    if (e == cudaSuccess && std::is_same<T, float>::value)
        e = cudaFuncSetAttribute(k_sor_rows_ens<T, BY, BZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)RowTile<T, BY, BZ>::smem());
    return e;
}

template <int BY, int BZ>
static void launch_rows_ens(const EnsTab<float>& tab, int in, int zero, int ctas, cudaStream_t s) {
    k_sor_rows_ens<float, BY, BZ><<<ctas, 256, RowTile<float, BY, BZ>::smem(), s>>>(tab, in, zero);
}

int launch_sor_ens(const EnsTab<float>& tab, int in, int zero, int ctas, cudaStream_t s) {
    switch (tab.tile) {
        case 0: launch_rows_ens<8, 8>(tab, in, zero, ctas, s); break;
        case 1: launch_rows_ens<4, 8>(tab, in, zero, ctas, s); break;
        case 2: launch_rows_ens<8, 4>(tab, in, zero, ctas, s); break;
        case 3: launch_rows_ens<16, 4>(tab, in, zero, ctas, s); break;
        default: launch_rows_ens<4, 16>(tab, in, zero, ctas, s); break;
    }
    return 1;
}

int ens_rows_smem(int t) {
    switch (t) {
        case 0: return (int)RowTile<float, 8, 8>::smem();
        case 1: return (int)RowTile<float, 4, 8>::smem();
        case 2: return (int)RowTile<float, 8, 4>::smem();
        case 3: return (int)RowTile<float, 16, 4>::smem();
        default: return (int)RowTile<float, 4, 16>::smem();
    }
}

template <typename T, int BY, int BZ>
static void launch_rows(const Geo<T>& g, const T* din, T* dout, const T* r, int zero_start, const Scalars* sc,
                        cudaStream_t s) {
    const Dom& d = g.d;
    dim3 grid((d.nx + 27) / 28, (d.ny + BY - 1) / BY, (d.nz + BZ - 1) / BZ);
    k_sor_rows<T, BY, BZ><<<grid, 256, RowTile<T, BY, BZ>::smem(), s>>>(g, din, dout, r, zero_start, sc);
}

template <typename T, int BX, int BY, int BZ>
constexpr size_t block_smem() {
    return sizeof(T) * ((BX + 4) * (BY + 4) * (BZ + 4) + (BX + 2) * (BY + 2) * (BZ + 2)) +
           (BX + 2) * (BY + 2) * (BZ + 2);
}

template <typename T, int BX, int BY, int BZ>
static cudaError_t allow_block() {
    return cudaFuncSetAttribute(k_sor_block<T, BX, BY, BZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)block_smem<T, BX, BY, BZ>());
}

template <typename T, int BX, int BY, int BZ>
static void launch_block(const Geo<T>& g, const T* din, T* dout, const T* r, int zero_start, const Scalars* sc,
                         cudaStream_t s) {
    const Dom& d = g.d;
    constexpr size_t bytes = block_smem<T, BX, BY, BZ>();
    dim3 grid((d.nx + BX - 1) / BX, (d.ny + BY - 1) / BY, (d.nz + BZ - 1) / BZ);
    k_sor_block<T, BX, BY, BZ><<<grid, 256, bytes, s>>>(g, din, dout, r, zero_start, sc);
}

template <typename T, int TX, int TY>
static void launch_tile(const Geo<T>& g, const T* din, T* dout, const T* r, int zero_start, const Scalars* sc,
                        int kc, cudaStream_t s) {
    const Dom& d = g.d;
    dim3 grid((d.nx + TX - 1) / TX, (d.ny + TY - 1) / TY, (d.nz + kc - 1) / kc);
    k_sor_fused<T, TX, TY><<<grid, TX / 2 * TY, 0, s>>>(g, din, dout, r, zero_start, sc, kc);
}

// tile shapes the autotuner chooses from: (TX, TY, 0) k-marching column tiles
// (the k-chunk is free), (BX, BY, BZ) 3-D blocks
const SorTile kSorTiles[] = {{32, 4, 0}, {32, 8, 0}, {64, 4, 0},  {64, 8, 0}, {128, 2, 0}, {128, 4, 0},
                             {32, 8, 4}, {32, 4, 8}, {64, 4, 4},  {32, 8, 8}, {16, 8, 8}, {64, 8, 2},
                             {28, 8, 8}, {28, 4, 8}, {28, 8, 4}, {28, 16, 4}, {28, 4, 16}};
const int kNumSorTiles = sizeof(kSorTiles) / sizeof(kSorTiles[0]);

// row-tile shape of ensemble tile index t (the row tiles of kSorTiles)
SorTile ens_tile_shape(int t) { return kSorTiles[kFirstRowTile + t]; }

template <typename T>
int launch_sor_fused(const Geo<T>& g, const T* din, T* dout, const T* r, int zero_start, const Scalars* sc,
                     SorCfg cfg, cudaStream_t s) {
    const int kc = cfg.kc > 0 ? cfg.kc : g.d.nz;
    switch (cfg.tile) {
        case 0: launch_tile<T, 32, 4>(g, din, dout, r, zero_start, sc, kc, s); break;
        case 1: launch_tile<T, 32, 8>(g, din, dout, r, zero_start, sc, kc, s); break;
        case 2: launch_tile<T, 64, 4>(g, din, dout, r, zero_start, sc, kc, s); break;
        case 3: launch_tile<T, 64, 8>(g, din, dout, r, zero_start, sc, kc, s); break;
        case 4: launch_tile<T, 128, 2>(g, din, dout, r, zero_start, sc, kc, s); break;
        case 5: launch_tile<T, 128, 4>(g, din, dout, r, zero_start, sc, kc, s); break;
        case 6: launch_block<T, 32, 8, 4>(g, din, dout, r, zero_start, sc, s); break;
        case 7: launch_block<T, 32, 4, 8>(g, din, dout, r, zero_start, sc, s); break;
        case 8: launch_block<T, 64, 4, 4>(g, din, dout, r, zero_start, sc, s); break;
        case 9: launch_block<T, 32, 8, 8>(g, din, dout, r, zero_start, sc, s); break;
        case 10: launch_block<T, 16, 8, 8>(g, din, dout, r, zero_start, sc, s); break;
        case 11: launch_block<T, 64, 8, 2>(g, din, dout, r, zero_start, sc, s); break;
        case 12: launch_rows<T, 8, 8>(g, din, dout, r, zero_start, sc, s); break;
        case 13: launch_rows<T, 4, 8>(g, din, dout, r, zero_start, sc, s); break;
        case 14: launch_rows<T, 8, 4>(g, din, dout, r, zero_start, sc, s); break;
        case 15: launch_rows<T, 16, 4>(g, din, dout, r, zero_start, sc, s); break;
        default: launch_rows<T, 4, 16>(g, din, dout, r, zero_start, sc, s); break;
    }
    return 1;
}

// opt the 3-D block kernels in to their dynamic shared memory on the current
// device (called when a handle is created, outside any stream capture)
template <typename T>
cudaError_t sor_prepare() {
    cudaError_t e = cudaSuccess, x;
    if ((x = allow_block<T, 32, 8, 4>()) != cudaSuccess) e = x;
    if ((x = allow_block<T, 32, 4, 8>()) != cudaSuccess) e = x;
    if ((x = allow_block<T, 64, 4, 4>()) != cudaSuccess) e = x;
    if ((x = allow_block<T, 32, 8, 8>()) != cudaSuccess) e = x;
    if ((x = allow_block<T, 16, 8, 8>()) != cudaSuccess) e = x;
    if ((x = allow_block<T, 64, 8, 2>()) != cudaSuccess) e = x;
    if ((x = allow_rows<T, 8, 8>()) != cudaSuccess) e = x;
    if ((x = allow_rows<T, 4, 8>()) != cudaSuccess) e = x;
    if ((x = allow_rows<T, 8, 4>()) != cudaSuccess) e = x;
    if ((x = allow_rows<T, 16, 4>()) != cudaSuccess) e = x;
    if ((x = allow_rows<T, 4, 16>()) != cudaSuccess) e = x;
    return e;
}
template cudaError_t sor_prepare<float>();
template cudaError_t sor_prepare<double>();

template int launch_sor_fused<float>(const Geo<float>&, const float*, float*, const float*, int, const Scalars*,
                                     SorCfg, cudaStream_t);
template int launch_sor_fused<double>(const Geo<double>&, const double*, double*, const double*, int,
                                      const Scalars*, SorCfg, cudaStream_t);

}  // namespace les
