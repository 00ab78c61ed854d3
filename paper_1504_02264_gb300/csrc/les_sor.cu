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

template <typename T, int TX, int TY>
static void launch_tile(const Geo<T>& g, const T* din, T* dout, const T* r, int zero_start, const Scalars* sc,
                        int kc, cudaStream_t s) {
    const Dom& d = g.d;
    dim3 grid((d.nx + TX - 1) / TX, (d.ny + TY - 1) / TY, (d.nz + kc - 1) / kc);
    k_sor_fused<T, TX, TY><<<grid, TX / 2 * TY, 0, s>>>(g, din, dout, r, zero_start, sc, kc);
}

// tile shapes the autotuner chooses from (TX, TY); the k-chunk is free
const SorTile kSorTiles[] = {{32, 4}, {32, 8}, {64, 4}, {64, 8}, {128, 2}, {128, 4}};
const int kNumSorTiles = sizeof(kSorTiles) / sizeof(kSorTiles[0]);

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
        default: launch_tile<T, 128, 4>(g, din, dout, r, zero_start, sc, kc, s); break;
    }
    return 1;
}

template int launch_sor_fused<float>(const Geo<float>&, const float*, float*, const float*, int, const Scalars*,
                                     SorCfg, cudaStream_t);
template int launch_sor_fused<double>(const Geo<double>&, const double*, double*, const double*, int,
                                      const Scalars*, SorCfg, cudaStream_t);

}  // namespace les
