// CUDA kernels of one LES time step (sm_103a), templated on the field type
// (float for the production path, double for bit-level parity checks).
//
// Routine map (paper Sec. 2.1): k_bc_* = bondv1, k_nut = les (eddy
// viscosity), k_momentum = velfg + les (SGS divergence) + adam + feedbf,
// k_outflow = bondv1 outflow and mass-flux correction, k_rhs / k_sor_half /
// k_accum / k_residual64 = press (Sec. 2.6), k_project = velnw.
#include <type_traits>

#include "les_internal.cuh"
#include "les_tma.cuh"

namespace les {

// ---------------------------------------------------------------------------
// counter-based inflow noise: splitmix64 as a hash of (seed, counter)
// (Steele, Lea & Flood 2014), then Box-Muller, in FP64.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t ctr) {
    uint64_t z = seed + (ctr + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double unit_open(uint64_t x) {
    return ((double)(x >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}
__device__ double gauss_at(uint64_t seed, uint64_t c) {
    double u1 = unit_open(splitmix64_at(seed, 2ull * c));
    double u2 = unit_open(splitmix64_at(seed, 2ull * c + 1ull));
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// ---------------------------------------------------------------------------
// bondv1, three passes (x over interior j,k; y over all i; z over all i,j) so
// corner ghosts take the rules in that order.

// inflow profile at level k of the current step: the fixed profile, or the
// series interpolated linearly in t = step * dt between the two bracketing
// profiles (held constant before the first and after the last)
__device__ __forceinline__ double inflow_at(const double* inflow, const InflowSeries& ser, long long step, int k,
                                            int nz) {
    if (ser.n <= 0) return inflow[k];
    const int sk = nz + 2, n = ser.n;
    const double t = (double)step * ser.dt;
    if (n == 1 || t <= ser.t[0]) return ser.p[k];
    if (t >= ser.t[n - 1]) return ser.p[(size_t)(n - 1) * sk + k];
    int m = 0;
    while (m + 1 < n - 1 && ser.t[m + 1] <= t) ++m;
    const double wgt = (t - ser.t[m]) / (ser.t[m + 1] - ser.t[m]);
    return (1.0 - wgt) * ser.p[(size_t)m * sk + k] + wgt * ser.p[(size_t)(m + 1) * sk + k];
}

template <typename T>
__global__ void k_bc_x(Dom d, T* u, T* v, T* w, const double* inflow, InflowSeries ser, double turb, uint64_t seed,
                       const Scalars* sc) {
    int j = blockIdx.x * blockDim.x + threadIdx.x + 1;
    int k = blockIdx.y + 1;
    if (j > d.ny) return;
    const int nx = d.nx;
    if (d.perx) {
        u[d.at(0, j, k)] = u[d.at(nx, j, k)];
        u[d.at(nx + 1, j, k)] = u[d.at(1, j, k)];
        v[d.at(0, j, k)] = v[d.at(nx, j, k)];
        v[d.at(nx + 1, j, k)] = v[d.at(1, j, k)];
        w[d.at(0, j, k)] = w[d.at(nx, j, k)];
        w[d.at(nx + 1, j, k)] = w[d.at(1, j, k)];
        return;
    }
    const double U = inflow_at(inflow, ser, sc->step, k, d.nz);
    double xu = 0.0, xv = 0.0, xw = 0.0;
    if (turb != 0.0) {
        const uint64_t sy = (uint64_t)(d.ny + 2), sz = (uint64_t)(d.nz + 2);
        uint64_t base = (uint64_t)sc->step * 3ull;
        xu = gauss_at(seed, ((base + 0) * sy + (uint64_t)j) * sz + (uint64_t)k);
        xv = gauss_at(seed, ((base + 1) * sy + (uint64_t)j) * sz + (uint64_t)k);
        xw = gauss_at(seed, ((base + 2) * sy + (uint64_t)j) * sz + (uint64_t)k);
    }
    u[d.at(0, j, k)] = (T)(U * (1.0 + turb * xu));
    v[d.at(0, j, k)] = (T)(turb * U * xv);
    w[d.at(0, j, k)] = (T)(turb * U * xw);
    T t = u[d.at(nx - 1, j, k)];
    u[d.at(nx, j, k)] = t;
    u[d.at(nx + 1, j, k)] = t;
    v[d.at(nx + 1, j, k)] = v[d.at(nx, j, k)];
    w[d.at(nx + 1, j, k)] = w[d.at(nx, j, k)];
}

template <typename T>
__global__ void k_bc_y(Dom d, T* u, T* v, T* w) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int k = blockIdx.y + 1;
    if (i > d.nx + 1) return;
    const int ny = d.ny;
    if (d.pery) {
        u[d.at(i, 0, k)] = u[d.at(i, ny, k)];
        u[d.at(i, ny + 1, k)] = u[d.at(i, 1, k)];
        v[d.at(i, 0, k)] = v[d.at(i, ny, k)];
        v[d.at(i, ny + 1, k)] = v[d.at(i, 1, k)];
        w[d.at(i, 0, k)] = w[d.at(i, ny, k)];
        w[d.at(i, ny + 1, k)] = w[d.at(i, 1, k)];
        return;
    }
    v[d.at(i, 0, k)] = T(0);
    v[d.at(i, ny, k)] = T(0);
    v[d.at(i, ny + 1, k)] = -v[d.at(i, ny - 1, k)];
    u[d.at(i, 0, k)] = u[d.at(i, 1, k)];
    u[d.at(i, ny + 1, k)] = u[d.at(i, ny, k)];
    w[d.at(i, 0, k)] = w[d.at(i, 1, k)];
    w[d.at(i, ny + 1, k)] = w[d.at(i, ny, k)];
}

template <typename T>
__global__ void k_bc_z(Dom d, T* u, T* v, T* w) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i > d.nx + 1) return;
    const int nz = d.nz;
    if (d.perz) {
        u[d.at(i, j, 0)] = u[d.at(i, j, nz)];
        u[d.at(i, j, nz + 1)] = u[d.at(i, j, 1)];
        v[d.at(i, j, 0)] = v[d.at(i, j, nz)];
        v[d.at(i, j, nz + 1)] = v[d.at(i, j, 1)];
        w[d.at(i, j, 0)] = w[d.at(i, j, nz)];
        w[d.at(i, j, nz + 1)] = w[d.at(i, j, 1)];
        return;
    }
    w[d.at(i, j, 0)] = T(0);
    w[d.at(i, j, nz)] = T(0);
    w[d.at(i, j, nz + 1)] = -w[d.at(i, j, nz - 1)];
    u[d.at(i, j, 0)] = -u[d.at(i, j, 1)];
    u[d.at(i, j, nz + 1)] = u[d.at(i, j, nz)];
    v[d.at(i, j, 0)] = -v[d.at(i, j, 1)];
    v[d.at(i, j, nz + 1)] = v[d.at(i, j, nz)];
}

template <typename T>
int launch_bc(const Geo<T>& g, T* u, T* v, T* w, const double* inflow, const InflowSeries& ser, double turb,
              uint64_t seed, const Scalars* sc, cudaStream_t s) {
    const Dom& d = g.d;
    k_bc_x<T><<<dim3((d.ny + 127) / 128, d.nz), 128, 0, s>>>(d, u, v, w, inflow, ser, turb, seed, sc);
    k_bc_y<T><<<dim3((d.nx + 2 + 127) / 128, d.nz), 128, 0, s>>>(d, u, v, w);
    k_bc_z<T><<<dim3((d.nx + 2 + 127) / 128, d.ny + 2), 128, 0, s>>>(d, u, v, w);
    return 3;
}

// ---------------------------------------------------------------------------
// les: Smagorinsky eddy viscosity at cell centres

// velocity reads around the cell (i0, j0, k0): the padded index of the cell
// once, neighbours by 32-bit offsets (rows and planes are < 2^31 elements)
// shear rates on cell edges, over any accessor D with U/V/W(i, j, k) and g
template <typename T, typename D>
struct StrainOps {
    __device__ __forceinline__ const D& self() const { return static_cast<const D&>(*this); }
    __device__ __forceinline__ T s12(int i, int j, int k) const {
        const D& S = self();
        return T(0.5) * ((S.U(i, j + 1, k) - S.U(i, j, k)) * S.g.rdy + (S.V(i + 1, j, k) - S.V(i, j, k)) * S.g.rdx);
    }
    __device__ __forceinline__ T s13(int i, int j, int k) const {
        const D& S = self();
        return T(0.5) * ((S.U(i, j, k + 1) - S.U(i, j, k)) * S.g.rdzs[k] + (S.W(i + 1, j, k) - S.W(i, j, k)) * S.g.rdx);
    }
    __device__ __forceinline__ T s23(int i, int j, int k) const {
        const D& S = self();
        return T(0.5) * ((S.V(i, j, k + 1) - S.V(i, j, k)) * S.g.rdzs[k] + (S.W(i, j + 1, k) - S.W(i, j, k)) * S.g.rdy);
    }
};

// nu_t ghost layer: zero gradient (the adjacent interior value) or periodic
// wrap, axis by axis (x over interior j, k; y over all i; z over all i, j), so
// a ghost read equals the read of the index clamped / wrapped on each axis
template <typename T>
__global__ void k_nut_ghost(Dom d, T* nut, int axis) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (axis == 0) {
        const int j = a + 1, k = b + 1;
        if (j > d.ny) return;
        nut[d.at(0, j, k)] = nut[d.at(d.perx ? d.nx : 1, j, k)];
        nut[d.at(d.nx + 1, j, k)] = nut[d.at(d.perx ? 1 : d.nx, j, k)];
    } else if (axis == 1) {
        const int i = a, k = b + 1;
        if (i > d.nx + 1) return;
        nut[d.at(i, 0, k)] = nut[d.at(i, d.pery ? d.ny : 1, k)];
        nut[d.at(i, d.ny + 1, k)] = nut[d.at(i, d.pery ? 1 : d.ny, k)];
    } else {
        const int i = a, j = b;
        if (i > d.nx + 1) return;
        nut[d.at(i, j, 0)] = nut[d.at(i, j, d.perz ? d.nz : 1)];
        nut[d.at(i, j, d.nz + 1)] = nut[d.at(i, j, d.perz ? 1 : d.nz)];
    }
}

// ---------------------------------------------------------------------------
// velfg + les (SGS) + adam + feedbf.  nu_t ghosts hold the clamped / wrapped
// values (k_nut_ghost), so the edge averages read it directly.

// nu_t averaged onto cell edges, over any accessor D with operator()(i, j, k)
template <typename T, typename D>
struct NutOps {
    __device__ __forceinline__ const D& self() const { return static_cast<const D&>(*this); }
    __device__ __forceinline__ T xy(int i, int j, int k) const {
        const D& N = self();
        return T(0.25) * (N(i, j, k) + N(i + 1, j, k) + N(i, j + 1, k) + N(i + 1, j + 1, k));
    }
    __device__ __forceinline__ T xz(int i, int j, int k) const {
        const D& N = self();
        return T(0.25) * (N(i, j, k) + N(i + 1, j, k) + N(i, j, k + 1) + N(i + 1, j, k + 1));
    }
    __device__ __forceinline__ T yz(int i, int j, int k) const {
        const D& N = self();
        return T(0.25) * (N(i, j, k) + N(i, j + 1, k) + N(i, j, k + 1) + N(i, j + 1, k + 1));
    }
};

// velocity and nu_t reads from a shared-memory window: planes in 4 rolling
// slots (plane k in slot k & 3), each MY rows of MX cells, the window's first
// cell being (ib, jb)
template <typename T, int MX, int MY>
struct SmemStencil : StrainOps<T, SmemStencil<T, MX, MY>> {
    const Geo<T>& g;
    const T* su;
    const T* sv;
    const T* sw;
    int ib, jb;
    __device__ __forceinline__ SmemStencil(const Geo<T>& g_, const T* su_, const T* sv_, const T* sw_, int ib_, int jb_)
        : g(g_), su(su_), sv(sv_), sw(sw_), ib(ib_), jb(jb_) {}
    __device__ __forceinline__ int at(int i, int j, int k) const { return ((k & 3) * MY + (j - jb)) * MX + (i - ib); }
    __device__ __forceinline__ T U(int i, int j, int k) const { return su[at(i, j, k)]; }
    __device__ __forceinline__ T V(int i, int j, int k) const { return sv[at(i, j, k)]; }
    __device__ __forceinline__ T W(int i, int j, int k) const { return sw[at(i, j, k)]; }
};

template <typename T, int MX, int MY>
struct SmemNut : NutOps<T, SmemNut<T, MX, MY>> {
    const T* sn;
    int ib, jb;
    __device__ __forceinline__ SmemNut(const T* sn_, int ib_, int jb_) : sn(sn_), ib(ib_), jb(jb_) {}
    __device__ __forceinline__ T operator()(int i, int j, int k) const {
        return sn[((k & 3) * MY + (j - jb)) * MX + (i - ib)];
    }
};

template <typename T, typename SA>
__device__ __forceinline__ T velfg_u(const Geo<T>& g, const SA& S, int i, int j, int k) {
    const T dx = g.dx, dy = g.dy, rdx = g.rdx, rdy = g.rdy;
    T um = S.U(i - 1, j, k), uc = S.U(i, j, k), up = S.U(i + 1, j, k);
    T cov1_i = T(0.5) * (um + uc) * (uc - um) * rdx;
    T cov1_ip = T(0.5) * (uc + up) * (up - uc) * rdx;
    T covx = (dx * cov1_i + dx * cov1_ip) * (T(0.5) * rdx);
    T vn = T(0.5) * (S.V(i, j, k) + S.V(i + 1, j, k));
    T vs = T(0.5) * (S.V(i, j - 1, k) + S.V(i + 1, j - 1, k));
    T un = S.U(i, j + 1, k), us = S.U(i, j - 1, k);
    T covy = (vs * (uc - us) * rdy + vn * (un - uc) * rdy) * T(0.5);
    T wt = T(0.5) * (S.W(i, j, k) + S.W(i + 1, j, k));
    T wb = T(0.5) * (S.W(i, j, k - 1) + S.W(i + 1, j, k - 1));
    T ut = S.U(i, j, k + 1), ub = S.U(i, j, k - 1);
    T covz = (wb * (uc - ub) * g.rdzs[k - 1] + wt * (ut - uc) * g.rdzs[k]) * T(0.5);
    T diu1_i = (uc - um) * rdx, diu1_ip = (up - uc) * rdx;
    T dfu = T(2) * (diu1_ip - diu1_i) * (T(0.5) * rdx) + ((un - uc) * rdy - (uc - us) * rdy) * rdy +
            ((ut - uc) * g.rdzs[k] - (uc - ub) * g.rdzs[k - 1]) * g.rdz[k];
    return -(covx + covy + covz) + g.nu * dfu;
}

template <typename T, typename SA>
__device__ __forceinline__ T velfg_v(const Geo<T>& g, const SA& S, int i, int j, int k) {
    const T dx = g.dx, dy = g.dy, rdx = g.rdx, rdy = g.rdy;
    T vm = S.V(i, j - 1, k), vc = S.V(i, j, k), vp = S.V(i, j + 1, k);
    T cov_j = T(0.5) * (vm + vc) * (vc - vm) * rdy;
    T cov_jp = T(0.5) * (vc + vp) * (vp - vc) * rdy;
    T covy = (dy * cov_j + dy * cov_jp) * (T(0.5) * rdy);
    T ue = T(0.5) * (S.U(i, j, k) + S.U(i, j + 1, k));
    T uw = T(0.5) * (S.U(i - 1, j, k) + S.U(i - 1, j + 1, k));
    T ve = S.V(i + 1, j, k), vw = S.V(i - 1, j, k);
    T covx = (uw * (vc - vw) * rdx + ue * (ve - vc) * rdx) * T(0.5);
    T wt = T(0.5) * (S.W(i, j, k) + S.W(i, j + 1, k));
    T wb = T(0.5) * (S.W(i, j, k - 1) + S.W(i, j + 1, k - 1));
    T vt = S.V(i, j, k + 1), vb = S.V(i, j, k - 1);
    T covz = (wb * (vc - vb) * g.rdzs[k - 1] + wt * (vt - vc) * g.rdzs[k]) * T(0.5);
    T dfv = ((ve - vc) * rdx - (vc - vw) * rdx) * rdx + T(2) * ((vp - vc) * rdy - (vc - vm) * rdy) * (T(0.5) * rdy) +
            ((vt - vc) * g.rdzs[k] - (vc - vb) * g.rdzs[k - 1]) * g.rdz[k];
    return -(covx + covy + covz) + g.nu * dfv;
}

template <typename T, typename SA>
__device__ __forceinline__ T velfg_w(const Geo<T>& g, const SA& S, int i, int j, int k) {
    const T dx = g.dx, dy = g.dy, rdx = g.rdx, rdy = g.rdy;
    const T dzk = g.dz[k], dzp = g.dz[k + 1], rdzk = g.rdz[k], rdzp = g.rdz[k + 1];
    const T rsum = T(1) / (dzk + dzp);
    T wm = S.W(i, j, k - 1), wc = S.W(i, j, k), wp = S.W(i, j, k + 1);
    T cov_k = T(0.5) * (wm + wc) * (wc - wm) * rdzk;
    T cov_kp = T(0.5) * (wc + wp) * (wp - wc) * rdzp;
    T covz = (dzp * cov_k + dzk * cov_kp) * rsum;
    T ue = (dzp * S.U(i, j, k) + dzk * S.U(i, j, k + 1)) * rsum;
    T uw = (dzp * S.U(i - 1, j, k) + dzk * S.U(i - 1, j, k + 1)) * rsum;
    T we = S.W(i + 1, j, k), ww = S.W(i - 1, j, k);
    T covx = (uw * (wc - ww) * rdx + ue * (we - wc) * rdx) * T(0.5);
    T vn = (dzp * S.V(i, j, k) + dzk * S.V(i, j, k + 1)) * rsum;
    T vs = (dzp * S.V(i, j - 1, k) + dzk * S.V(i, j - 1, k + 1)) * rsum;
    T wn = S.W(i, j + 1, k), wsv = S.W(i, j - 1, k);
    T covy = (vs * (wc - wsv) * rdy + vn * (wn - wc) * rdy) * T(0.5);
    T dfw = ((we - wc) * rdx - (wc - ww) * rdx) * rdx + ((wn - wc) * rdy - (wc - wsv) * rdy) * rdy +
            T(2) * ((wp - wc) * rdzp - (wc - wm) * rdzk) * rsum;
    return -(covx + covy + covz) + g.nu * dfw;
}

template <typename T, typename SA, typename NA>
__device__ __forceinline__ T sgs_u(const Geo<T>& g, const SA& S, const NA& N, int i,
                                        int j, int k) {
    T t11_i = T(2) * N(i, j, k) * (S.U(i, j, k) - S.U(i - 1, j, k)) * g.rdx;
    T t11_ip = T(2) * N(i + 1, j, k) * (S.U(i + 1, j, k) - S.U(i, j, k)) * g.rdx;
    T t12_n = T(2) * N.xy(i, j, k) * S.s12(i, j, k);
    T t12_s = T(2) * N.xy(i, j - 1, k) * S.s12(i, j - 1, k);
    T t13_t = T(2) * N.xz(i, j, k) * S.s13(i, j, k);
    T t13_b = T(2) * N.xz(i, j, k - 1) * S.s13(i, j, k - 1);
    return (t11_ip - t11_i) * g.rdx + (t12_n - t12_s) * g.rdy + (t13_t - t13_b) * g.rdz[k];
}
template <typename T, typename SA, typename NA>
__device__ __forceinline__ T sgs_v(const Geo<T>& g, const SA& S, const NA& N, int i,
                                        int j, int k) {
    T t22_j = T(2) * N(i, j, k) * (S.V(i, j, k) - S.V(i, j - 1, k)) * g.rdy;
    T t22_jp = T(2) * N(i, j + 1, k) * (S.V(i, j + 1, k) - S.V(i, j, k)) * g.rdy;
    T t12_e = T(2) * N.xy(i, j, k) * S.s12(i, j, k);
    T t12_w = T(2) * N.xy(i - 1, j, k) * S.s12(i - 1, j, k);
    T t23_t = T(2) * N.yz(i, j, k) * S.s23(i, j, k);
    T t23_b = T(2) * N.yz(i, j, k - 1) * S.s23(i, j, k - 1);
    return (t12_e - t12_w) * g.rdx + (t22_jp - t22_j) * g.rdy + (t23_t - t23_b) * g.rdz[k];
}
template <typename T, typename SA, typename NA>
__device__ __forceinline__ T sgs_w(const Geo<T>& g, const SA& S, const NA& N, int i,
                                        int j, int k) {
    T t33_k = T(2) * N(i, j, k) * (S.W(i, j, k) - S.W(i, j, k - 1)) * g.rdz[k];
    T t33_kp = T(2) * N(i, j, k + 1) * (S.W(i, j, k + 1) - S.W(i, j, k)) * g.rdz[k + 1];
    T t13_e = T(2) * N.xz(i, j, k) * S.s13(i, j, k);
    T t13_w = T(2) * N.xz(i - 1, j, k) * S.s13(i - 1, j, k);
    T t23_n = T(2) * N.yz(i, j, k) * S.s23(i, j, k);
    T t23_s = T(2) * N.yz(i, j - 1, k) * S.s23(i, j - 1, k);
    return (t13_e - t13_w) * g.rdx + (t23_n - t23_s) * g.rdy + (t33_kp - t33_k) * g.rdzs[k];
}

// Plane kk of NF fields for slot kk & 3 of their shared-memory windows (MY
// rows of MX cells from padded cell (ib, jb); zeros outside the padded box),
// in two halves: window_fetch issues the global loads into registers,
// window_put stores them, so a plane's loads can be in flight while the
// previous plane is computed.  Fixed trip counts keep everything in registers.
template <typename T, int NF, int MX, int MY, int NT>
struct Window {
    static constexpr int NP = MX * MY, REPS = (NP + NT - 1) / NT;
    T val[REPS][NF];
    __device__ __forceinline__ void fetch(const Dom& d, const T* const (&src)[NF], int ib, int jb, int kk, int tid) {
#pragma unroll
        for (int rep = 0; rep < REPS; ++rep) {
            const int q = tid + rep * NT;
            const int gi = ib + q % MX, gj = jb + q / MX;
            const bool in = q < NP && gi <= d.nx + 1 && gj <= d.ny + 1;
            const long long x = in ? d.at(gi, gj, kk) : 0;
#pragma unroll
            for (int f = 0; f < NF; ++f) val[rep][f] = in ? src[f][x] : T(0);
        }
    }
    __device__ __forceinline__ void put(T* const (&dst)[NF], int kk, int tid) const {
        const int o = (kk & 3) * NP;
#pragma unroll
        for (int rep = 0; rep < REPS; ++rep) {
            const int q = tid + rep * NT;
            if (q < NP)
#pragma unroll
                for (int f = 0; f < NF; ++f) dst[f][o + q] = val[rep][f];
        }
    }
};

// A CTA owns a 32 x 8 column of cells and marches up kc planes.  The planes
// k-1 .. k+1 of u, v, w and nu_t, each with a 1-cell ring, sit in shared
// memory in 4 rolling slots: plane k+1 goes to the slot that plane k-3 held,
// which no thread reads any more, so one barrier per plane suffices, and the
// loads of plane k+2 are in flight (in registers) while plane k is computed.  Every read of the per-cell formulas then hits shared memory
// (the previous one-thread-per-cell version waited on ~150 dependent global
// loads per cell).  The arithmetic is the per-cell formulas above, unchanged.
constexpr int kMomTX = 32, kMomTY = 8;

template <typename T>
__global__ void __launch_bounds__(kMomTX * kMomTY)
k_momentum(Geo<T> g, const T* __restrict__ u, const T* __restrict__ v, const T* __restrict__ w,
           const T* __restrict__ nut, T* __restrict__ fu, T* __restrict__ fv, T* __restrict__ fw, T* __restrict__ us,
           T* __restrict__ vs, T* __restrict__ ws, const Scalars* __restrict__ sc, int kc) {
    constexpr int MX = kMomTX + 2, MY = kMomTY + 2, NP = MX * MY, NT = kMomTX * kMomTY;
    __shared__ T sU[4 * NP], sV[4 * NP], sW[4 * NP], sN[4 * NP];
    const Dom& d = g.d;
    const bool first = sc->step == 0;
    const int tid = threadIdx.x + kMomTX * threadIdx.y;
    const int ib = blockIdx.x * kMomTX, jb = blockIdx.y * kMomTY;    // window corner (ring included)
    const int i = ib + 1 + threadIdx.x, j = jb + 1 + threadIdx.y;
    const int k0 = 1 + blockIdx.z * kc, k1 = min(k0 + kc, d.nz + 1);
    const T* const src[4] = {u, v, w, nut};
    T* const dst[4] = {sU, sV, sW, sN};
    Window<T, 4, MX, MY, NT> win;
    const SmemStencil<T, MX, MY> S(g, sU, sV, sW, ib, jb);
    const SmemNut<T, MX, MY> N(sN, ib, jb);
    win.fetch(d, src, ib, jb, k0 - 1, tid);
    win.put(dst, k0 - 1, tid);
    win.fetch(d, src, ib, jb, k0, tid);
    win.put(dst, k0, tid);
    win.fetch(d, src, ib, jb, k0 + 1, tid);
    const bool own = i <= d.nx && j <= d.ny;
    for (int k = k0; k < k1; ++k) {
        // the cell's own flags and previous tendencies, issued before the
        // barrier so that their latency overlaps it
        const long long c = own ? d.at(i, j, k) : 0;
        uint8_t f = 0;
        T fu0 = T(0), fv0 = T(0), fw0 = T(0);
        if (own) {
            f = g.flags[c];
            if (!first) {
                fu0 = fu[c];
                fv0 = fv[c];
                fw0 = fw[c];
            }
        }
        // plane k+1 into the slot plane k-3 held; plane k+2 in flight during plane k
        win.put(dst, k + 1, tid);
        __syncthreads();
        if (k + 2 <= k1) win.fetch(d, src, ib, jb, k + 2, tid);
        if (!own) continue;
        if (i <= (d.perx ? d.nx : d.nx - 1)) {
            T F = velfg_u(g, S, i, j, k) + sgs_u(g, S, N, i, j, k);
            T Fh = first ? F : T(1.5) * F - T(0.5) * fu0;
            fu[c] = F;
            us[c] = (f & F_E) ? S.U(i, j, k) + g.dt * Fh : T(0);
        }
        if (j <= (d.pery ? d.ny : d.ny - 1)) {
            T F = velfg_v(g, S, i, j, k) + sgs_v(g, S, N, i, j, k);
            T Fh = first ? F : T(1.5) * F - T(0.5) * fv0;
            fv[c] = F;
            vs[c] = (f & F_N) ? S.V(i, j, k) + g.dt * Fh : T(0);
        }
        if (k <= (d.perz ? d.nz : d.nz - 1)) {
            T F = velfg_w(g, S, i, j, k) + sgs_w(g, S, N, i, j, k);
            T Fh = first ? F : T(1.5) * F - T(0.5) * fw0;
            fw[c] = F;
            ws[c] = (f & F_T) ? S.W(i, j, k) + g.dt * Fh : T(0);
        }
    }
}

// les (Smagorinsky eddy viscosity at cell centres) on the same staged
// window: u, v, w planes k-1 .. k+1 with a 1-cell ring
template <typename T>
__global__ void __launch_bounds__(kMomTX * kMomTY)
k_nut(Geo<T> g, const T* __restrict__ u, const T* __restrict__ v, const T* __restrict__ w, T* __restrict__ nut,
      int kc) {
    constexpr int MX = kMomTX + 2, MY = kMomTY + 2, NP = MX * MY, NT = kMomTX * kMomTY;
    __shared__ T sU[4 * NP], sV[4 * NP], sW[4 * NP];
    const Dom& d = g.d;
    const int tid = threadIdx.x + kMomTX * threadIdx.y;
    const int ib = blockIdx.x * kMomTX, jb = blockIdx.y * kMomTY;
    const int i = ib + 1 + threadIdx.x, j = jb + 1 + threadIdx.y;
    const int k0 = 1 + blockIdx.z * kc, k1 = min(k0 + kc, d.nz + 1);
    const T* const src[3] = {u, v, w};
    T* const dst[3] = {sU, sV, sW};
    Window<T, 3, MX, MY, NT> win;
    const SmemStencil<T, MX, MY> S(g, sU, sV, sW, ib, jb);
    const bool own = i <= d.nx && j <= d.ny;
    win.fetch(d, src, ib, jb, k0 - 1, tid);
    win.put(dst, k0 - 1, tid);
    win.fetch(d, src, ib, jb, k0, tid);
    win.put(dst, k0, tid);
    win.fetch(d, src, ib, jb, k0 + 1, tid);
    for (int k = k0; k < k1; ++k) {
        const long long c = own ? d.at(i, j, k) : 0;
        const uint8_t f = own ? g.flags[c] : 0;
        win.put(dst, k + 1, tid);
        __syncthreads();
        if (k + 2 <= k1) win.fetch(d, src, ib, jb, k + 2, tid);
        if (!own) continue;
        if (!(f & F_FLUID)) {
            nut[c] = T(0);
            continue;
        }
        T s11 = (S.U(i, j, k) - S.U(i - 1, j, k)) * g.rdx;
        T s22 = (S.V(i, j, k) - S.V(i, j - 1, k)) * g.rdy;
        T s33 = (S.W(i, j, k) - S.W(i, j, k - 1)) * g.rdz[k];
        T s12 = T(0.25) * (S.s12(i - 1, j - 1, k) + S.s12(i, j - 1, k) + S.s12(i - 1, j, k) + S.s12(i, j, k));
        T s13 = T(0.25) * (S.s13(i - 1, j, k - 1) + S.s13(i, j, k - 1) + S.s13(i - 1, j, k) + S.s13(i, j, k));
        T s23 = T(0.25) * (S.s23(i, j - 1, k - 1) + S.s23(i, j, k - 1) + S.s23(i, j - 1, k) + S.s23(i, j, k));
        T smag = sqrt(T(2) * (s11 * s11 + s22 * s22 + s33 * s33) + T(4) * (s12 * s12 + s13 * s13 + s23 * s23));
        nut[c] = g.delta2[k] * smag;
    }
}

// planes per CTA: enough CTAs for a few waves on every SM, few ring planes
int momentum_kc(const Dom& d) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 132;
    }
    const long long cols = (long long)((d.nx + kMomTX - 1) / kMomTX) * ((d.ny + kMomTY - 1) / kMomTY);
    const long long target = (long long)sms * 24;
    const long long kc = (cols * d.nz + target - 1) / target;
    return (int)(kc < 4 ? 4 : (kc > 32 ? 32 : kc));
}

template <typename T>
int launch_nut(const Geo<T>& g, const T* u, const T* v, const T* w, T* nut, cudaStream_t s) {
    const Dom& d = g.d;
    const int kc = momentum_kc(d);
    k_nut<T><<<dim3((d.nx + kMomTX - 1) / kMomTX, (d.ny + kMomTY - 1) / kMomTY, (d.nz + kc - 1) / kc),
               dim3(kMomTX, kMomTY), 0, s>>>(g, u, v, w, nut, kc);
    k_nut_ghost<T><<<dim3((d.ny + 127) / 128, d.nz), 128, 0, s>>>(d, nut, 0);
    k_nut_ghost<T><<<dim3((d.nx + 2 + 127) / 128, d.nz), 128, 0, s>>>(d, nut, 1);
    k_nut_ghost<T><<<dim3((d.nx + 2 + 127) / 128, d.ny + 2), 128, 0, s>>>(d, nut, 2);
    return 4;
}

template <typename T>
int launch_momentum(const Geo<T>& g, const T* u, const T* v, const T* w, const T* nut, T* fu, T* fv,
                    T* fw, T* us, T* vs, T* ws, const Scalars* sc, cudaStream_t s) {
    const Dom& d = g.d;
    const int kc = momentum_kc(d);
    k_momentum<T><<<dim3((d.nx + kMomTX - 1) / kMomTX, (d.ny + kMomTY - 1) / kMomTY, (d.nz + kc - 1) / kc),
                    dim3(kMomTX, kMomTY), 0, s>>>(g, u, v, w, nut, fu, fv, fw, us, vs, ws, sc, kc);
    return 1;
}

// ---------------------------------------------------------------------------
// FP64 block reductions, deterministic for a fixed launch shape.  FP64
// arithmetic is narrow on this part (a warp-wide add queues for many cycles),
// so the values go to shared memory and one warp adds them: 8 sequential adds
// per lane and a 5-level shuffle tree, 13 warp-wide adds per value instead of
// a shuffle tree in every warp.  Blocks of at most 256 threads; the total is
// valid on thread 0.
constexpr int kSumThreads = 256;

template <int NV>
__device__ __forceinline__ void block_sum(double (&x)[NV]) {
    __shared__ double sh[NV][kSumThreads];
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nt = blockDim.x * blockDim.y;
    __syncthreads();          // a previous call's readers are done with sh
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[q][tid] = x[q];
    __syncthreads();
    if (tid < 32) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double v = 0.0;
            for (int m = tid; m < nt; m += 32) v += sh[q][m];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            x[q] = v;
        }
    }
}

// Each block stores its partial sums; the last block to finish adds all the
// partials in block order and returns true (with the totals in x on thread 0).
template <int NV>
__device__ bool grid_sum_at(double (&x)[NV], const Reduce& r, unsigned nb, unsigned b) {
    block_sum<NV>(x);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    __shared__ bool last;
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) r.partials[(size_t)q * nb + b] = x[q];
        __threadfence();
        unsigned t = atomicAdd(r.counter, 1u);
        last = (t == nb - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    const int nt = blockDim.x * blockDim.y;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        // four independent chains so that four loads are in flight
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        const double* pq = r.partials + (size_t)q * nb;
        unsigned m = tid;
        for (; m + 3 * nt < nb; m += 4 * nt) {
            s0 += __ldcg(&pq[m]);
            s1 += __ldcg(&pq[m + nt]);
            s2 += __ldcg(&pq[m + 2 * nt]);
            s3 += __ldcg(&pq[m + 3 * nt]);
        }
        for (; m < nb; m += nt) s0 += __ldcg(&pq[m]);
        x[q] = (s0 + s1) + (s2 + s3);
    }
    block_sum<NV>(x);
    if (tid == 0) *r.counter = 0u;
    return true;
}

template <int NV>
__device__ bool grid_sum(double (&x)[NV], const Reduce& r) {
    return grid_sum_at<NV>(x, r, gridDim.x * gridDim.y * gridDim.z,
                           blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z));
}

// ---------------------------------------------------------------------------
// bondv1 on u*: inflow face copied, zero-gradient outflow, FP64 mass-flux
// correction (one block; the plane is small), periodic face copies.

// inflow face copied into u*, inflow and outflow fluxes summed (FP64, last
// block), the correction factor stored; periodic x: the face copy only
template <typename T>
__global__ void k_outflow_sum(Geo<T> g, const T* u, T* us, Reduce red) {
    const Dom& d = g.d;
    const int n = d.ny * d.nz;
    const int q0 = blockIdx.x * blockDim.x + threadIdx.x, qs = gridDim.x * blockDim.x;
    if (d.perx) {        // uniform over the grid
        for (int q = q0; q < n; q += qs) {
            const int j = q % d.ny + 1, k = q / d.ny + 1;
            us[d.at(0, j, k)] = us[d.at(d.nx, j, k)];
        }
        if (q0 == 0) {
            red.sc->mass_factor = 1.0;
            red.sc->q_in = red.sc->q_out = 0.0;
        }
        return;
    }
    double x[2] = {0.0, 0.0};
    for (int q = q0; q < n; q += qs) {
        const int j = q % d.ny + 1, k = q / d.ny + 1;
        const T ui = u[d.at(0, j, k)];
        const T uo = us[d.at(d.nx - 1, j, k)];
        us[d.at(0, j, k)] = ui;
        x[0] += (double)ui * (double)g.dy * g.dz64[k];
        x[1] += (double)uo * (double)g.dy * g.dz64[k];
    }
    if (grid_sum<2>(x, red) && threadIdx.x == 0) {
        Scalars* sc = red.sc;
        const double f = fabs(x[1]) > 1e-300 ? x[0] / x[1] : 1.0;
        sc->mass_factor = f;
        sc->q_in = x[0];
        sc->q_out = x[1] * f;
    }
}

// zero-gradient outflow scaled by the mass-flux correction
template <typename T>
__global__ void k_outflow_apply(Geo<T> g, T* us, const Scalars* sc) {
    const Dom& d = g.d;
    if (d.perx) return;
    const int n = d.ny * d.nz;
    const double f = sc->mass_factor;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const int j = q % d.ny + 1, k = q / d.ny + 1;
        us[d.at(d.nx, j, k)] = (T)((double)us[d.at(d.nx - 1, j, k)] * f);
    }
}

template <typename T>
__global__ void k_wrap_faces(Dom d, T* vs, T* ws, int zaxis) {
    int a = blockIdx.x * blockDim.x + threadIdx.x + 1;
    int b = blockIdx.y + 1;
    if (a > d.nx) return;
    if (!zaxis) vs[d.at(a, 0, b)] = vs[d.at(a, d.ny, b)];     // periodic y: a = i, b = k
    else ws[d.at(a, b, 0)] = ws[d.at(a, b, d.nz)];            // periodic z: a = i, b = j
}

template <typename T>
int launch_outflow(const Geo<T>& g, const T* u, T* us, T* vs, T* ws, const Reduce& red, cudaStream_t s) {
    const Dom& d = g.d;
    const int n_face = d.ny * d.nz;
    const int nb = n_face < 64 * 256 ? (n_face + 255) / 256 : 64;
    k_outflow_sum<T><<<nb, 256, 0, s>>>(g, u, us, red);
    k_outflow_apply<T><<<nb, 256, 0, s>>>(g, us, red.sc);
    int n = 2;
    if (d.pery) {
        k_wrap_faces<T><<<dim3((d.nx + 127) / 128, d.nz), 128, 0, s>>>(d, vs, ws, 0);
        n++;
    }
    if (d.perz) {
        k_wrap_faces<T><<<dim3((d.nx + 127) / 128, d.ny), 128, 0, s>>>(d, vs, ws, 1);
        n++;
    }
    return n;
}

// ---------------------------------------------------------------------------
// press: rhs = div(u*)/dt on fluid cells; FP64 dz-weighted mean (last block)

// Column kernels with a grid reduction: each thread walks kc planes of its
// (i, j) column, kc chosen so that at most ~8192 CTAs leave partial sums for
// the last block to add (one CTA per plane left it ~10^5 partials on large
// grids).
int column_kc(const Dom& d) {
    const long long cols = (long long)((d.nx + 31) / 32) * ((d.ny + 7) / 8);
    const long long kc = (cols * d.nz + 8191) / 8192;
    return (int)(kc < 1 ? 1 : (kc > d.nz ? d.nz : kc));
}

template <typename T>
__global__ void k_rhs(Geo<T> g, const T* us, const T* vs, const T* ws, T* rhs, double vfluid, Reduce r, int kc) {
    const Dom& d = g.d;
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    const int kb = blockIdx.z * kc + 1, ke = min(kb + kc, d.nz + 1);
    double x[1] = {0.0};
    if (i <= d.nx && j <= d.ny) {
        long long c = d.at(i, j, kb);
        for (int k = kb; k < ke; ++k, c += d.plane) {
            T val = T(0);
            if (g.flags[c] & F_FLUID) {
                T div = (us[c] - us[c - 1]) / g.dx + (vs[c] - vs[c - d.px]) / g.dy +
                        (ws[c] - ws[c - d.plane]) / g.dz[k];
                val = div / g.dt;
                x[0] += g.dz64[k] * (double)val;
            }
            rhs[c] = val;
        }
    }
    if (grid_sum<1>(x, r)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) r.sc->rhs_mean = vfluid > 0.0 ? x[0] / vfluid : 0.0;
    }
}

// FP32 fields: a thread takes 4 consecutive cells of a row with 16-byte
// loads and stores (a padded row starts 16-byte aligned and cell i = 1 sits
// 16 bytes into it, so cells 1 + 4t .. 4 + 4t are aligned), a CTA of 32 x 8
// threads a 128 x 8 column tile over kc planes, two planes' loads in flight
// at a time; the bottom face of a plane is the top face of the previous one,
// kept in registers.  The per-cell arithmetic is that of k_rhs.
struct RhsPlane {
    uchar4 f;
    float4 ue, vn, vsth, wt;
    float uw;
};
__device__ __forceinline__ void rhs_load(const Geo<float>& g, const float* __restrict__ us,
                                         const float* __restrict__ vs, const float* __restrict__ ws, long long c,
                                         RhsPlane& P) {
    P.f = *reinterpret_cast<const uchar4*>(g.flags + c);
    P.ue = *reinterpret_cast<const float4*>(us + c);
    P.uw = us[c - 1];
    P.vn = *reinterpret_cast<const float4*>(vs + c);
    P.vsth = *reinterpret_cast<const float4*>(vs + c - g.d.px);
    P.wt = *reinterpret_cast<const float4*>(ws + c);
}
__global__ void __launch_bounds__(256) k_rhs4(Geo<float> g, const float* __restrict__ us, const float* __restrict__ vs,
                                              const float* __restrict__ ws, float* __restrict__ rhs, double vfluid,
                                              Reduce r, int kc) {
    const Dom& d = g.d;
    const int i = (blockIdx.x * 32 + threadIdx.x) * 4 + 1;
    const int j = blockIdx.y * 8 + threadIdx.y + 1;
    const int kb = blockIdx.z * kc + 1, ke = min(kb + kc, d.nz + 1);
    double x[1] = {0.0};
    if (i <= d.nx && j <= d.ny) {
        const int ne = min(4, d.nx + 1 - i);             // cells of this thread inside the grid
        long long c = d.at(i, j, kb);
        float4 wb = *reinterpret_cast<const float4*>(ws + c - d.plane);
        auto plane = [&](const RhsPlane& P, int k, long long cc) {
            const uint8_t fl[4] = {P.f.x, P.f.y, P.f.z, P.f.w};
            const float ue[4] = {P.ue.x, P.ue.y, P.ue.z, P.ue.w}, uw[4] = {P.uw, P.ue.x, P.ue.y, P.ue.z};
            const float vn[4] = {P.vn.x, P.vn.y, P.vn.z, P.vn.w}, vsh[4] = {P.vsth.x, P.vsth.y, P.vsth.z, P.vsth.w};
            const float wt[4] = {P.wt.x, P.wt.y, P.wt.z, P.wt.w}, wbb[4] = {wb.x, wb.y, wb.z, wb.w};
            float val[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                val[e] = 0.f;
                if (e < ne && (fl[e] & F_FLUID)) {
                    const float div = (ue[e] - uw[e]) / g.dx + (vn[e] - vsh[e]) / g.dy + (wt[e] - wbb[e]) / g.dz[k];
                    val[e] = div / g.dt;
                    x[0] += g.dz64[k] * (double)val[e];
                }
            }
            if (ne == 4) {
                *reinterpret_cast<float4*>(rhs + cc) = make_float4(val[0], val[1], val[2], val[3]);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (e < ne) rhs[cc + e] = val[e];
            }
            wb = P.wt;
        };
        int k = kb;
        for (; k + 1 < ke; k += 2, c += 2 * d.plane) {
            RhsPlane A, B;
            rhs_load(g, us, vs, ws, c, A);
            rhs_load(g, us, vs, ws, c + d.plane, B);
            plane(A, k, c);
            plane(B, k + 1, c + d.plane);
        }
        if (k < ke) {
            RhsPlane A;
            rhs_load(g, us, vs, ws, c, A);
            plane(A, k, c);
        }
    }
    if (grid_sum<1>(x, r)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) r.sc->rhs_mean = vfluid > 0.0 ? x[0] / vfluid : 0.0;
    }
}

template <typename T>
int launch_rhs(const Geo<T>& g, const T* us, const T* vs, const T* ws, T* rhs, double vfluid,
               const Reduce& r, cudaStream_t s) {
    const Dom& d = g.d;
    if constexpr (std::is_same<T, float>::value) {
        // about 4096 CTAs (a few waves), at most one per plane of a column
        // tile (the size of the reduction's partials array)
        const long long cols = (long long)((d.nx + 127) / 128) * ((d.ny + 7) / 8);
        long long kc = (cols * d.nz + 4095) / 4096;
        kc = kc < 1 ? 1 : (kc > d.nz ? d.nz : kc);
        k_rhs4<<<dim3((d.nx + 127) / 128, (d.ny + 7) / 8, (d.nz + (int)kc - 1) / (int)kc), dim3(32, 8), 0, s>>>(
            g, us, vs, ws, rhs, vfluid, r, (int)kc);
    } else {
        const int kc = column_kc(d);
        k_rhs<T><<<dim3((d.nx + 31) / 32, (d.ny + 7) / 8, (d.nz + kc - 1) / kc), dim3(32, 8), 0, s>>>(
            g, us, vs, ws, rhs, vfluid, r, kc);
    }
    return 1;
}

// caller-supplied rhs: zero non-fluid cells and compute the mean
template <typename T>
__global__ void k_rhs_mean(Geo<T> g, T* rhs, double vfluid, Reduce r, int kc) {
    const Dom& d = g.d;
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    const int kb = blockIdx.z * kc + 1, ke = min(kb + kc, d.nz + 1);
    double x[1] = {0.0};
    if (i <= d.nx && j <= d.ny) {
        long long c = d.at(i, j, kb);
        for (int k = kb; k < ke; ++k, c += d.plane) {
            if (g.flags[c] & F_FLUID) x[0] += g.dz64[k] * (double)rhs[c];
            else rhs[c] = T(0);
        }
    }
    if (grid_sum<1>(x, r)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) r.sc->rhs_mean = vfluid > 0.0 ? x[0] / vfluid : 0.0;
    }
}

template <typename T>
int launch_rhs_mean(const Geo<T>& g, T* rhs, double vfluid, const Reduce& r, cudaStream_t s) {
    const Dom& d = g.d;
    const int kc = column_kc(d);
    k_rhs_mean<T><<<dim3((d.nx + 31) / 32, (d.ny + 7) / 8, (d.nz + kc - 1) / kc), dim3(32, 8), 0, s>>>(
        g, rhs, vfluid, r, kc);
    return 1;
}

// ---------------------------------------------------------------------------
// press: red-black SOR (Sec. 2.6) as mixed-precision iterative refinement.
//
// The pressure p is kept in FP64.  Each batch of sweeps runs the printed SOR
// update in the field type T on the correction d, A d = r, from d = 0, where
// r = (rhs - mean) - A p is formed in FP64.  SOR is a linear stationary
// iteration, so p + d after m sweeps equals m plain SOR sweeps on p in exact
// arithmetic; keeping p in FP64 removes the FP32 residual floor.

template <typename T>
struct Poisson {
    const Geo<T>& g;
    template <typename R>
    __device__ __forceinline__ void coefs(uint8_t f, int k, R cx, R cy, const R* cT, const R* cB, R& ae, R& aw,
                                          R& an, R& as, R& at, R& ab) const {
        ae = (f & F_E) ? cx : R(0);
        aw = (f & F_W) ? cx : R(0);
        an = (f & F_N) ? cy : R(0);
        as = (f & F_S) ? cy : R(0);
        at = (f & F_T) ? cT[k] : R(0);
        ab = (f & F_B) ? cB[k] : R(0);
    }
    // neighbour indices (wrapped on periodic axes)
    __device__ __forceinline__ void nbr(int i, int j, int k, long long& e, long long& w, long long& n,
                                        long long& s, long long& t, long long& b) const {
        const Dom& d = g.d;
        int ie = (d.perx && i == d.nx) ? 1 : i + 1;
        int iw = (d.perx && i == 1) ? d.nx : i - 1;
        int jn = (d.pery && j == d.ny) ? 1 : j + 1;
        int js = (d.pery && j == 1) ? d.ny : j - 1;
        int kt = (d.perz && k == d.nz) ? 1 : k + 1;
        int kb = (d.perz && k == 1) ? d.nz : k - 1;
        e = d.at(ie, j, k);
        w = d.at(iw, j, k);
        n = d.at(i, jn, k);
        s = d.at(i, js, k);
        t = d.at(i, j, kt);
        b = d.at(i, j, kb);
    }
};

// One half-sweep on the correction d (in place; a colour reads only the other
// colour).  zero_start: first sweep of a batch, d = 0 everywhere before it.
template <typename T>
__global__ void k_sor_half(Geo<T> g, T* dl, const T* r, int nrd, int zero_arg, const Scalars* sc) {
    const Dom& d = g.d;
    if (sc->done) return;
    const bool zero_start = zero_arg == 1 || (zero_arg == 2 && sc->zflag);
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    int k = blockIdx.z + 1;
    if (j > d.ny) return;
    int i = 1 + ((k + j + nrd) & 1) + 2 * m;
    if (i > d.nx) return;
    long long c = d.at(i, j, k);
    const uint8_t f = g.flags[c];
    if (!(f & F_UNK)) return;
    Poisson<T> P{g};
    T ae, aw, an, as, at, ab;
    P.coefs(f, k, g.cx, g.cy, g.cT, g.cB, ae, aw, an, as, at, ab);
    T cn1 = T(1) / (ae + aw + an + as + at + ab);
    long long e, w, n, s_, t, b;
    P.nbr(i, j, k, e, w, n, s_, t, b);
    T s = T(0);
    const bool nb_zero = zero_start && nrd == 0;   // red reads black, still zero
    if (!nb_zero) {
        s += ae * dl[e];
        s += aw * dl[w];
        s += an * dl[n];
        s += as * dl[s_];
        s += at * dl[t];
        s += ab * dl[b];
    }
    T own = zero_start ? T(0) : dl[c];
    T reltmp = g.omega * (cn1 * (s - r[c]) - own);
    dl[c] = own + reltmp;
}

template <typename T>
int launch_sor_sweep(const Geo<T>& g, T* dl, const T* r, int zero_start, const Scalars* sc, cudaStream_t s) {
    const Dom& d = g.d;
    dim3 grid(((d.nx + 1) / 2 + 31) / 32, (d.ny + 7) / 8, d.nz);
    k_sor_half<T><<<grid, dim3(32, 8), 0, s>>>(g, dl, r, 0, zero_start, sc);
    k_sor_half<T><<<grid, dim3(32, 8), 0, s>>>(g, dl, r, 1, zero_start, sc);
    return 2;
}

// Refinement: ph += d on the unknowns (own cell only, so in place).
// kc planes from plane bz * kc + 1 of a 32 x 8 column tile
template <typename T>
__device__ __forceinline__ void accum_body(const Geo<T>& g, double* ph, const T* dl, int bx, int by, int bz,
                                           int kc = 1) {
    const Dom& d = g.d;
    const int i = bx * blockDim.x + threadIdx.x + 1;
    const int j = by * blockDim.y + threadIdx.y + 1;
    const int kb = bz * kc + 1, ke = min(kb + kc, d.nz + 1);
    if (i > d.nx || j > d.ny) return;
    long long c = d.at(i, j, kb);
    for (int k = kb; k < ke; ++k, c += d.plane)
        if (g.flags[c] & F_UNK) ph[c] += (double)dl[c];
}

template <typename T>
__global__ void k_accum(Geo<T> g, double* ph, const T* dl, const Scalars* sc, int gate, int kc) {
    pdl_wait();
    if (gate && (sc->done || !sc->refine)) return;
    accum_body<T>(g, ph, dl, blockIdx.x, blockIdx.y, blockIdx.z, kc);
}

// planes per thread of the accumulation: about 8 CTAs per SM, so that a
// launch gated off (no refinement asked for) costs little
int accum_kc(const Dom& d) {
    const long long cols = (long long)((d.nx + 31) / 32) * ((d.ny + 7) / 8);
    const long long kc = (cols * d.nz + 1215) / 1216;
    return (int)(kc < 1 ? 1 : (kc > d.nz ? d.nz : kc));
}

template <typename T>
int launch_accum(const Geo<T>& g, double* ph, const T* dl, const Scalars* sc, int gate, cudaStream_t s) {
    const Dom& d = g.d;
    const int kc = accum_kc(d);
    launch_pdl(k_accum<T>, dim3((d.nx + 31) / 32, (d.ny + 7) / 8, (d.nz + kc - 1) / kc), dim3(32, 8), 0, s, g, ph,
               dl, sc, gate, kc);
    return 1;
}

// Grid-stride reductions use at most kReduceBlocks blocks, so the last-block
// completion counter sees few atomics.
constexpr int kReduceBlocks = 1024;
int reduce_blocks(const Dom& d) {
    long long n = (long long)d.nx * d.ny * d.nz;
    long long b = (n + 255) / 256;
    return (int)(b < kReduceBlocks ? b : kReduceBlocks);
}

__device__ __forceinline__ void cell_of(const Dom& d, int q, int& i, int& j, int& k) {
    i = q % d.nx + 1;
    const int t = q / d.nx;
    j = t % d.ny + 1;
    k = t / d.ny + 1;
}

// r = (rhs - mean) - A ph formed in FP64 and stored in T; FP64 norms, the
// true relative residual and stop test, the dz-weighted fluid mean of ph (for
// the gauge) and the bookkeeping of the SOR loop in the last block.
// block b of nb (grid-stride over the cells); returns, on thread 0 of the
// last block, 1 if this residual ended the solve, else 0 (-1 elsewhere)
template <typename T>
__device__ __forceinline__ int residual64_body(const Geo<T>& g, const double* ph, const T* rhs, T* r,
                                               double vfluid, const Reduce& red, const CondArgs& ca, unsigned b,
                                               unsigned nb) {
    const Dom& d = g.d;
    const int n = d.nx * d.ny * d.nz;
    const double mean = red.sc->rhs_mean;
    const bool init = ca.mode == RES_INIT;
    const int nt = blockDim.x * blockDim.y, tid = threadIdx.x + blockDim.x * threadIdx.y;    // 1-D or 32 x 8
    double x[3] = {0.0, 0.0, 0.0};
    for (int q = b * nt + tid; q < n; q += nb * nt) {
        int i, j, k;
        cell_of(d, q, i, j, k);
        long long c = d.at(i, j, k);
        const uint8_t f = g.flags[c];
        const double pc = ph[c];
        if (f & F_UNK) {
            Poisson<T> Q{g};
            double ae, aw, an, as, at, ab;
            Q.coefs(f, k, g.cx64, g.cy64, g.cT64, g.cB64, ae, aw, an, as, at, ab);
            long long e, w, nn, s_, t, b;
            Q.nbr(i, j, k, e, w, nn, s_, t, b);
            double s = 0.0;
            s += ae * ph[e];
            s += aw * ph[w];
            s += an * ph[nn];
            s += as * ph[s_];
            s += at * ph[t];
            s += ab * ph[b];
            // the coefficient sum from the table: the same FP64 sum, off the
            // narrow FP64 pipe
            const double diag = g.diag64[k * 64 + (f & 63)];
            const double bb = (double)rhs[c] - mean;
            const double res = bb - (s - diag * pc);
            r[c] = (T)res;
            x[0] += res * res;
            if (init) x[1] += bb * bb;      // |b| is fixed for the solve: summed once, at its start
        }
        if (f & F_FLUID) x[2] += g.dz64[k] * pc;
    }
    if (grid_sum_at<3>(x, red, nb, b)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            Scalars* sc = red.sc;
            sc->res2 = x[0];
            if (init) sc->rhs2 = x[1];
            const double rhs2 = sc->rhs2;
            const double rel = rhs2 == 0.0 ? sqrt(x[0]) : sqrt(x[0] / rhs2);
            const bool conv = rel <= ca.tol;
            const bool bad = !isfinite(rel);
            sc->rel = rel;
            sc->converged = conv;
            sc->nonfinite = bad;
            sc->p_mean = vfluid > 0.0 ? x[2] / vfluid : 0.0;
            sc->rho_ref = rel;
            sc->since = 0;
            sc->zflag = 1;
            sc->refine = 0;
            int done = 0;
            if (ca.mode == RES_INIT) {
                sc->sweeps = 0;
                sc->batches = 0;
            } else if (ca.mode == RES_LOOP) {
                sc->batches += 1;
                done = conv || bad || sc->sweeps >= ca.limit;
                if (done && !conv) sc->noconv_any = 1;
            } else {
                sc->sweeps += ca.n;
                sc->batches += 1;
                done = 1;
            }
            sc->done = done;
            if (ca.done_host) *(volatile int*)ca.done_host = done;
            return done;
        }
    }
    return -1;
}

template <typename T>
__global__ void __launch_bounds__(256) k_residual64(Geo<T> g, const double* ph, const T* rhs, T* r, double vfluid,
                                                    Reduce red, CondArgs ca) {
    pdl_wait();
    if (ca.gate == 1 && (red.sc->done || !red.sc->refine)) return;     // uniform over the grid
    if (ca.gate == 2 && red.sc->done) return;
    residual64_body<T>(g, ph, rhs, r, vfluid, red, ca, blockIdx.x, gridDim.x);
}

template <typename T>
int launch_residual64(const Geo<T>& g, const double* ph, const T* rhs, T* r, double vfluid, const Reduce& red,
                      CondArgs ca, cudaStream_t s) {
    launch_pdl(k_residual64<T>, dim3(reduce_blocks(g.d)), dim3(256), 0, s, g, ph, rhs, r, vfluid, red, ca);
    return 1;
}

// Cheap convergence estimate after a batch of sweeps: e = r - A d in the field
// type (difference form sum a_nb (d_nb - d_c), no cancellation against the
// diagonal), |e| / |rhs| with FP64 sums.  b - A(p + d) = r - A d exactly, so
// this is the residual of the current iterate up to rounding.  It only decides
// when to take the FP64 refinement, which makes the stop decision.
// the estimate's bookkeeping from the grid's sum of squared residuals (one
// thread): the relative estimate, the sweep counters and whether a
// refinement is due
__device__ __forceinline__ void est_finish(double sum, const Reduce& red, const CondArgs& ca) {
    Scalars* sc = red.sc;
    const double rhs2 = sc->rhs2;
    const double est = rhs2 == 0.0 ? sqrt(sum) : sqrt(sum / rhs2);
    sc->est = est;
    sc->sweeps += ca.n;
    sc->since += ca.n;
    sc->zflag = 0;
    const bool need = ca.force || !(est > ca.tol) || est <= kRefineDrop * sc->rho_ref ||
                      sc->since >= kRefineEvery || sc->sweeps >= ca.limit;
    sc->refine = need;
}

template <typename T>
__device__ __forceinline__ void sor_est_body(const Geo<T>& g, const T* __restrict__ dl, const T* __restrict__ r,
                                             T* __restrict__ rout, const Reduce& red, const CondArgs& ca, int bx,
                                             int by, int bz, unsigned nb, unsigned b) {
    const Dom& d = g.d;
    // a (32 x 8) column tile over a chunk of kEstChunk planes, unrolled: the
    // chunk's flags first, then every load of the chunk before its use (the
    // padded array holds every neighbour, so the loads need no face test);
    // neighbour offsets are 32-bit
    const int i = bx * 32 + threadIdx.x + 1;
    const int j = by * 8 + threadIdx.y + 1;
    const int kb = bz * kEstChunk + 1, ke = min(kb + kEstChunk, d.nz + 1);
    T acc = T(0);
    if (i <= d.nx && j <= d.ny) {
        const int pl = (int)d.plane;
        const int oe = (d.perx && i == d.nx) ? -(d.nx - 1) : 1;
        const int ow = (d.perx && i == 1) ? (d.nx - 1) : -1;
        const int on = (d.pery && j == d.ny) ? -(d.ny - 1) * d.px : d.px;
        const int os = (d.pery && j == 1) ? (d.ny - 1) * d.px : -d.px;
        const long long c0 = d.at(i, j, kb);
        uint8_t fl[kEstChunk];
#pragma unroll
        for (int m = 0; m < kEstChunk; ++m) fl[m] = kb + m < ke ? g.flags[c0 + (long long)m * pl] : (uint8_t)0;
        // half a chunk at a time, every load of the half issued before its
        // use (unconditionally: the padded array holds each neighbour; a
        // plane past the chunk reads the chunk's first plane)
        constexpr int H = kEstChunk / 2;
#pragma unroll
        for (int h = 0; h < kEstChunk; h += H) {
            T dc[H], de[H], dw[H], dn[H], ds[H], dt[H], db[H], rc[H];
#pragma unroll
            for (int q = 0; q < H; ++q) {
                const int m = h + q, k = kb + m;
                const long long c = k < ke ? c0 + (long long)m * pl : c0;
                const int kk = k < ke ? k : kb;
                const int ot = (d.perz && kk == d.nz) ? -(d.nz - 1) * pl : pl;
                const int ob = (d.perz && kk == 1) ? (d.nz - 1) * pl : -pl;
                dc[q] = dl[c];
                de[q] = dl[c + oe];
                dw[q] = dl[c + ow];
                dn[q] = dl[c + on];
                ds[q] = dl[c + os];
                dt[q] = dl[c + ot];
                db[q] = dl[c + ob];
                rc[q] = r[c];
            }
#pragma unroll
            for (int q = 0; q < H; ++q) {
                const int m = h + q;
                const uint8_t f = fl[m];
                if (!(f & F_UNK)) continue;
                const int k = kb + m;
                T s = T(0);
                if (f & F_E) s += g.cx * (de[q] - dc[q]);
                if (f & F_W) s += g.cx * (dw[q] - dc[q]);
                if (f & F_N) s += g.cy * (dn[q] - dc[q]);
                if (f & F_S) s += g.cy * (ds[q] - dc[q]);
                if (f & F_T) s += g.cT[k] * (dt[q] - dc[q]);
                if (f & F_B) s += g.cB[k] * (db[q] - dc[q]);
                const T res = rc[q] - s;
                if (rout) rout[c0 + (long long)m * pl] = res;   // the current residual, input of the network correction
                acc += res * res;
            }
        }
    }
    double x[1] = {(double)acc};
    if (grid_sum_at<1>(x, red, nb, b))
        if (threadIdx.x == 0 && threadIdx.y == 0) est_finish(x[0], red, ca);
}

// (FP32: at most 64 registers, four CTAs per SM: the half-chunk loads alone would
// take 80 and three CTAs; the learned step measured 0.6% faster so)
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2)
    k_sor_est(Geo<T> g, const T* dl, const T* r, T* rout, Reduce red, CondArgs ca) {
    pdl_wait();
    if (red.sc->done) return;      // uniform over the grid
    sor_est_body<T>(g, dl, r, rout, red, ca, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x * gridDim.y * gridDim.z,
                    blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z));
}

template <typename T>
int launch_sor_est(const Geo<T>& g, const T* dl, const T* r, T* rout, const Reduce& red, CondArgs ca,
                   cudaStream_t s) {
    const Dom& d = g.d;
    dim3 grid((d.nx + 31) / 32, (d.ny + 7) / 8, (d.nz + kEstChunk - 1) / kEstChunk);
    launch_pdl(k_sor_est<T>, grid, dim3(32, 8), 0, s, g, dl, r, rout, red, ca);
    return 1;
}

// The same estimate on an FP32 grid with no periodic axis, its loads from
// three TMA tile copies instead of eight global loads per cell: a CTA's
// 32 x 8 x kEstChunk cells with d on a 1-cell ring (40 x 10 x 10 box from the
// padded column of i0 - 4), r on the cells, the flags (48 wide from the
// 16-byte column at or below that of i0 - 4).  Each thread takes the same
// cells in the same order with the same arithmetic, and the block and grid
// sums are those of k_sor_est (same launch shape), so the result is the same.
//
// With S > 0 (S = 4 or 8) the CTA also forms the network's pooled input for
// its cells, which the stride-S cubes tile exactly: the residual and the
// unknown mask summed over each cube with the pooling kernel's sums in its
// order (k_pool_rms: the same pooled values), scaled by 1/S^3, and each
// cube's m r^2 and m added to the grid sums next to the residual's, so that
// the last block also leaves the mask-weighted RMS and the mask sum (FP64,
// summed in this kernel's fixed block order).
template <int S>
__global__ void __launch_bounds__(256, S > 0 ? 6 : 4)
    k_sor_est_tma(const __grid_constant__ CUtensorMap td, const __grid_constant__ CUtensorMap tr,
                  const __grid_constant__ CUtensorMap tf, Geo<float> g, float* __restrict__ rout, Reduce red,
                  CondArgs ca, EstPool pool) {
    static_assert(kEstChunk == 8, "tile boxes of 8 planes");
    static_assert(S == 0 || S == 4 || S == 8, "pooling strides that tile the 32 x 8 x 8 block");
    __shared__ __align__(128) float sD[kEstChunk + 2][10][40];
    __shared__ __align__(128) float sR[kEstChunk][8][32];
    __shared__ __align__(128) uint8_t sF[kEstChunk][8][48];
    __shared__ __align__(8) uint64_t bar_word;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
    const uint32_t bar = tma::smem_u32(&bar_word);
    const Dom& d = g.d;
    const int i0 = blockIdx.x * 32 + 1, j0 = blockIdx.y * 8 + 1, kb = blockIdx.z * kEstChunk + 1;
    // the kernel before this one is a sweep, which writes only d: r and the
    // flags are copied before the dependency wait, d after it
    if (tid == 0) {
        tma::mbar_init(bar, 1);
        tma::mbar_fence_init();
        tma::mbar_expect_tx_only(bar, (uint32_t)(sizeof(sR) + sizeof(sF)));
        tma::tma_load_3d(tma::smem_u32(sR), &tr, 32 * blockIdx.x + 4, j0, kb, bar);
        tma::tma_load_3d(tma::smem_u32(sF), &tf, 32 * blockIdx.x, j0, kb, bar);
    }
    pdl_wait();
    if (tid == 0) {
        tma::mbar_expect_tx(bar, (uint32_t)sizeof(sD));
        tma::tma_load_3d(tma::smem_u32(sD), &td, 32 * blockIdx.x, j0 - 1, kb - 1, bar);
    }
    if (red.sc->done) {            // uniform over the grid: let the copies land (bounded), then leave
        if (tid == 0) tma::mbar_wait_bounded(bar, 0u);
        __syncthreads();
        return;
    }
    bool ok = true;
    if (tid == 0) {
        ok = tma::mbar_wait_bounded(bar, 0u);
        if (!ok) {
            atomicExch(&red.sc->timeout, 1);
            tma::mbar_wait_bounded(bar, 0u);      // copies still in flight: a bounded chance to land
        }
    }
    ok = __syncthreads_and(ok);
    float acc = 0.f;
    unsigned umask = 0;                            // bit m: plane m's cell is an unknown of the grid
    const int i = i0 + tx, j = j0 + ty;
    if (ok && i <= d.nx && j <= d.ny) {
        const int ke = min(kb + kEstChunk, d.nz + 1);
        const long long c0 = d.at(i, j, kb);
        const long long pl = d.plane;
#pragma unroll
        for (int m = 0; m < kEstChunk; ++m) {
            if (kb + m >= ke) break;
            const uint8_t f = sF[m][ty][tx + 4];
            if (!(f & F_UNK)) continue;
            const int k = kb + m;
            const float dc = sD[m + 1][ty + 1][tx + 4];
            float s = 0.f;
            if (f & F_E) s += g.cx * (sD[m + 1][ty + 1][tx + 5] - dc);
            if (f & F_W) s += g.cx * (sD[m + 1][ty + 1][tx + 3] - dc);
            if (f & F_N) s += g.cy * (sD[m + 1][ty + 2][tx + 4] - dc);
            if (f & F_S) s += g.cy * (sD[m + 1][ty][tx + 4] - dc);
            if (f & F_T) s += g.cT[k] * (sD[m + 2][ty + 1][tx + 4] - dc);
            if (f & F_B) s += g.cB[k] * (sD[m][ty + 1][tx + 4] - dc);
            const float res = sR[m][ty][tx] - s;
            if (rout) rout[c0 + m * pl] = res;
            acc += res * res;
            if constexpr (S > 0) {
                sR[m][ty][tx] = res;       // no other thread reads this entry
                umask |= 1u << m;
            }
        }
    }
    double x[S > 0 ? 3 : 1];
    x[0] = (double)acc;
    if constexpr (S > 0) {
        // the residual (stored above) and the mask of the block's cells over
        // r's and the flags' tiles (each thread writes only the entries it
        // read; six CTAs per SM, as many as the plain estimate's registers give);
        // then the pooling kernel's sums in its order: per cube, for each of
        // SZ z-offsets p and S rows q, the cells of planes p, p + SZ, ... of
        // row q along x (into the d tile, read by no one any more), then
        // those partials with p outer and q inner
        constexpr int SZ = S < 4 ? S : 4;
        constexpr int NXC = 32 / S, NYC = 8 / S, NZC = kEstChunk / S, NCUBE = NXC * NYC * NZC;
        constexpr int NPART = NCUBE * SZ * S;
        static_assert(2 * NPART <= (int)(sizeof(sD) / sizeof(float)) && NCUBE <= 256, "pooling scratch");
#pragma unroll
        for (int m = 0; m < kEstChunk; ++m) {
            const bool u = (umask >> m) & 1u;
            if (!u) sR[m][ty][tx] = 0.f;
            sF[m][ty][tx + 4] = u ? 1 : 0;
        }
        __syncthreads();
        float* partr = &sD[0][0][0];
        float* partm = partr + NPART;
        for (int q = tid; q < NPART; q += 256) {
            const int row = q % S, pz = (q / S) % SZ, cube = q / (S * SZ);
            const int cx = cube % NXC, fy = (cube / NXC) % NYC * S + row, fz0 = cube / (NXC * NYC) * S + pz;
            float ar = 0.f, am = 0.f;
#pragma unroll
            for (int zz = 0; zz < S; zz += SZ)
#pragma unroll
                for (int e = 0; e < S; ++e) {
                    ar += sR[fz0 + zz][fy][cx * S + e];
                    am += (float)sF[fz0 + zz][fy][cx * S + e + 4];
                }
            partr[q] = ar;
            partm[q] = am;
        }
        __syncthreads();
        x[1] = 0.0;
        x[2] = 0.0;
        if (tid < NCUBE) {
            const int cx = tid % NXC, cy = (tid / NXC) % NYC, cz = tid / (NXC * NYC);
            float tr = 0.f, tm = 0.f;
#pragma unroll
            for (int q = 0; q < SZ * S; ++q) {
                tr += partr[tid * SZ * S + q];
                tm += partm[tid * SZ * S + q];
            }
            const int gx = blockIdx.x * NXC + cx, gy = blockIdx.y * NYC + cy, gz = blockIdx.z * NZC + cz;
            if (gx < pool.xc && gy < pool.yc && gz < pool.zc) {
                const float inv = 1.f / (float)(S * S * S);
                const float vr = tr * inv, vm = tm * inv;
                const long long v = ((long long)gz * pool.yc + gy) * pool.xc + gx;
                pool.rc[v] = vr;
                pool.mask[v] = vm;
                x[1] = (double)vm * (double)vr * (double)vr;
                x[2] = (double)vm;
            }
        }
    }
    if (grid_sum<(S > 0 ? 3 : 1)>(x, red))
        if (tid == 0) {
            est_finish(x[0], red, ca);
            if constexpr (S > 0) {
                pool.scal[0] = x[2] > 0.0 ? sqrt(x[1] / x[2]) : 0.0;
                pool.scal[1] = x[2];
            }
        }
}

int launch_sor_est_tma(const Geo<float>& g, const CUtensorMap* maps4, int dcur, float* rout, const Reduce& red,
                       CondArgs ca, cudaStream_t s, const EstPool& pool) {
    const Dom& d = g.d;
    dim3 grid((d.nx + 31) / 32, (d.ny + 7) / 8, (d.nz + kEstChunk - 1) / kEstChunk);
    if (pool.rc && pool.s == 8)
        launch_pdl(k_sor_est_tma<8>, grid, dim3(32, 8), 0, s, maps4[dcur], maps4[2], maps4[3], g, rout, red, ca, pool);
    else if (pool.rc && pool.s == 4)
        launch_pdl(k_sor_est_tma<4>, grid, dim3(32, 8), 0, s, maps4[dcur], maps4[2], maps4[3], g, rout, red, ca, pool);
    else
        launch_pdl(k_sor_est_tma<0>, grid, dim3(32, 8), 0, s, maps4[dcur], maps4[2], maps4[3], g, rout, red, ca, pool);
    return 1;
}

// ---------------------------------------------------------------------------
// velnw: gauge (p -= dz-weighted fluid mean) and u = u* - dt grad p, the
// gradient taken in FP64 from the FP64 pressure.  Reads ph_in, writes the
// gauged pressure to ph_out (no in-place race).

template <typename T>
__global__ void k_project(Geo<T> g, const T* us, const T* vs, const T* ws, T* u, T* v, T* w,
                          const double* ph_in, double* ph_out, Scalars* sc) {
    const Dom& d = g.d;
    int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    int k = blockIdx.z + 1;
    // the step counter advances here, after every reader of it has run
    if (i == 1 && j == 1 && k == 1) sc->step += 1;
    if (i > d.nx || j > d.ny) return;
    long long c = d.at(i, j, k);
    const uint8_t f = g.flags[c];
    const double pm = sc->p_mean;
    if constexpr (std::is_same<T, float>::value) {
        // FP32 fields: an open face joins two fluid cells, so the gauge cancels
        // in the pressure difference; the difference is taken in FP64 (no
        // cancellation error) and the rest of the update in FP32, which keeps
        // this kernel off GB300's narrow FP64 pipe (no FP64 division)
        const double praw = ph_in[c];
        ph_out[c] = (f & F_FLUID) ? praw - pm : praw;
        if (i <= (d.perx ? d.nx : d.nx - 1)) {
            const int ie = (d.perx && i == d.nx) ? 1 : i + 1;
            const float val = (f & F_E) ? us[c] - (g.dt * g.rdx) * (float)(ph_in[d.at(ie, j, k)] - praw) : 0.f;
            u[c] = val;
            if (d.perx && i == d.nx) u[d.at(0, j, k)] = val;
        } else {
            u[c] = us[c];
        }
        if (!d.perx && i == 1) u[d.at(0, j, k)] = us[d.at(0, j, k)];
        if (j <= (d.pery ? d.ny : d.ny - 1)) {
            const int jn = (d.pery && j == d.ny) ? 1 : j + 1;
            const float val = (f & F_N) ? vs[c] - (g.dt * g.rdy) * (float)(ph_in[d.at(i, jn, k)] - praw) : 0.f;
            v[c] = val;
            if (d.pery && j == d.ny) v[d.at(i, 0, k)] = val;
        } else {
            v[c] = vs[c];
        }
        if (!d.pery && j == 1) v[d.at(i, 0, k)] = vs[d.at(i, 0, k)];
        if (k <= (d.perz ? d.nz : d.nz - 1)) {
            const int kt = (d.perz && k == d.nz) ? 1 : k + 1;
            const float val = (f & F_T) ? ws[c] - (g.dt * g.rdzs[k]) * (float)(ph_in[d.at(i, j, kt)] - praw) : 0.f;
            w[c] = val;
            if (d.perz && k == d.nz) w[d.at(i, j, 0)] = val;
        } else {
            w[c] = ws[c];
        }
        if (!d.perz && k == 1) w[d.at(i, j, 0)] = ws[d.at(i, j, 0)];
        return;
    }
    const double dt = (double)g.dt;
    auto gp = [&](long long q) -> double { return (g.flags[q] & F_FLUID) ? ph_in[q] - pm : ph_in[q]; };
    const double pc = gp(c);
    ph_out[c] = pc;
    // u on the east face of cell i
    if (i <= (d.perx ? d.nx : d.nx - 1)) {
        int ie = (d.perx && i == d.nx) ? 1 : i + 1;
        T val = (f & F_E) ? (T)((double)us[c] - dt * (gp(d.at(ie, j, k)) - pc) / g.dx64) : T(0);
        u[c] = val;
        if (d.perx && i == d.nx) u[d.at(0, j, k)] = val;
    } else {
        u[c] = us[c];
    }
    if (!d.perx && i == 1) u[d.at(0, j, k)] = us[d.at(0, j, k)];
    // v on the north face of cell j
    if (j <= (d.pery ? d.ny : d.ny - 1)) {
        int jn = (d.pery && j == d.ny) ? 1 : j + 1;
        T val = (f & F_N) ? (T)((double)vs[c] - dt * (gp(d.at(i, jn, k)) - pc) / g.dy64) : T(0);
        v[c] = val;
        if (d.pery && j == d.ny) v[d.at(i, 0, k)] = val;
    } else {
        v[c] = vs[c];
    }
    if (!d.pery && j == 1) v[d.at(i, 0, k)] = vs[d.at(i, 0, k)];
    // w on the top face of cell k
    if (k <= (d.perz ? d.nz : d.nz - 1)) {
        int kt = (d.perz && k == d.nz) ? 1 : k + 1;
        T val = (f & F_T) ? (T)((double)ws[c] - dt * (gp(d.at(i, j, kt)) - pc) / g.dzs64[k]) : T(0);
        w[c] = val;
        if (d.perz && k == d.nz) w[d.at(i, j, 0)] = val;
    } else {
        w[c] = ws[c];
    }
    if (!d.perz && k == 1) w[d.at(i, j, 0)] = ws[d.at(i, j, 0)];
}

template <typename T>
int launch_project(const Geo<T>& g, const T* us, const T* vs, const T* ws, T* u, T* v, T* w,
                   const double* ph_in, double* ph_out, Scalars* sc, cudaStream_t s) {
    const Dom& d = g.d;
    k_project<T><<<dim3((d.nx + 31) / 32, (d.ny + 7) / 8, d.nz), dim3(32, 8), 0, s>>>(
        g, us, vs, ws, u, v, w, ph_in, ph_out, sc);
    return 1;
}

// gauge alone (les_pressure_solve): p_out = p_in - dz-weighted fluid mean
template <typename T>
__global__ void k_gauge(Geo<T> g, const double* p_in, double* p_out, const Scalars* sc) {
    const Dom& d = g.d;
    int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    int k = blockIdx.z + 1;
    if (i > d.nx || j > d.ny) return;
    long long c = d.at(i, j, k);
    p_out[c] = (g.flags[c] & F_FLUID) ? p_in[c] - sc->p_mean : p_in[c];
}

template <typename T>
int launch_gauge(const Geo<T>& g, const double* p_in, double* p_out, const Scalars* sc, cudaStream_t s) {
    const Dom& d = g.d;
    k_gauge<T><<<dim3((d.nx + 31) / 32, (d.ny + 7) / 8, d.nz), dim3(32, 8), 0, s>>>(g, p_in, p_out, sc);
    return 1;
}

// mean-removed rhs for inspection
template <typename T>
__global__ void k_rhs_eff(Geo<T> g, const T* rhs, T* out, const Scalars* sc) {
    const Dom& d = g.d;
    int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    int k = blockIdx.z + 1;
    if (i > d.nx || j > d.ny) return;
    long long c = d.at(i, j, k);
    out[c] = (g.flags[c] & F_FLUID) ? rhs[c] - (T)sc->rhs_mean : T(0);
}

template <typename T>
int launch_rhs_eff(const Geo<T>& g, const T* rhs, T* out, const Scalars* sc, cudaStream_t s) {
    const Dom& d = g.d;
    k_rhs_eff<T><<<dim3((d.nx + 31) / 32, (d.ny + 7) / 8, d.nz), dim3(32, 8), 0, s>>>(g, rhs, out, sc);
    return 1;
}

// ---------------------------------------------------------------------------
// learned warm start support: line search and update along a predicted
// correction (dense (nz, ny, nx) array), plus recording of training pairs.

// alpha minimising the energy norm of the error along q (FP64):
//   alpha = <q, V r> / <q, V A q>,  V = diag(dz_k) (the cell volumes up to dx dy),
// which makes V A symmetric, so this is the exact minimiser of
// (e - alpha q)^T (-V A) (e - alpha q) with A e = r.  Smooth predictions with
// some high-frequency noise keep a useful step (the residual-norm minimiser
// <r, A q> / <A q, A q> would be dominated by A's amplified noise).
// The step needs only moderate precision (it decides the efficiency of the
// correction, not the solution), so A q and the per-thread sums are formed in
// the field type and the grid sums in FP64.  Tiles of (32 x 8) columns march
// over kEstChunk planes, like the estimate.
template <typename T>
__global__ void __launch_bounds__(256) k_warm_ls(Geo<T> g, const T* __restrict__ r, const float* __restrict__ q,
                                                 double* alpha, Reduce red,
                                                 int in_loop) {
    pdl_wait();
    const Dom& d = g.d;
    if (red.sc->done) return;      // uniform over the grid
    if (in_loop == 2 && !red.sc->qpend) return;
    const int i = blockIdx.x * 32 + threadIdx.x + 1;
    const int j = blockIdx.y * 8 + threadIdx.y + 1;
    const int kb = blockIdx.z * kEstChunk + 1, ke = min(kb + kEstChunk, d.nz + 1);
    T s0 = T(0), s1 = T(0);
    if (i <= d.nx && j <= d.ny) {
        // dense offsets (the grid has < 2^31 cells); flags never open a face
        // across a non-periodic domain boundary, so every neighbour read
        // stays inside the dense array.  The chunk is unrolled: its flags
        // first, then its loads, then the sums.
        const int sy = d.nx, sz = d.nx * d.ny;
        const int oe = (d.perx && i == d.nx) ? -(d.nx - 1) : 1;
        const int ow = (d.perx && i == 1) ? (d.nx - 1) : -1;
        const int on = (d.pery && j == d.ny) ? -(d.ny - 1) * sy : sy;
        const int os = (d.pery && j == 1) ? (d.ny - 1) * sy : -sy;
        const int pl = (int)d.plane;
        const long long c0 = d.at(i, j, kb);
        const int v0 = ((kb - 1) * d.ny + (j - 1)) * d.nx + (i - 1);
        uint8_t fl[kEstChunk];
#pragma unroll
        for (int m = 0; m < kEstChunk; ++m) fl[m] = kb + m < ke ? g.flags[c0 + (long long)m * pl] : (uint8_t)0;
#pragma unroll
        for (int m = 0; m < kEstChunk; ++m) {
            const uint8_t f = fl[m];
            if (!(f & F_UNK)) continue;
            const int k = kb + m;
            const long long c = c0 + (long long)m * pl;
            const int v = v0 + m * sz;
            const int ot = (d.perz && k == d.nz) ? -(d.nz - 1) * sz : sz;
            const int ob = (d.perz && k == 1) ? (d.nz - 1) * sz : -sz;
            const T qc = (T)q[v], rc = r[c];
            const T qe = (f & F_E) ? (T)q[v + oe] : T(0), qw = (f & F_W) ? (T)q[v + ow] : T(0);
            const T qn = (f & F_N) ? (T)q[v + on] : T(0), qs = (f & F_S) ? (T)q[v + os] : T(0);
            const T qt = (f & F_T) ? (T)q[v + ot] : T(0), qb = (f & F_B) ? (T)q[v + ob] : T(0);
            T aq = T(0);
            if (f & F_E) aq += g.cx * (qe - qc);
            if (f & F_W) aq += g.cx * (qw - qc);
            if (f & F_N) aq += g.cy * (qn - qc);
            if (f & F_S) aq += g.cy * (qs - qc);
            if (f & F_T) aq += g.cT[k] * (qt - qc);
            if (f & F_B) aq += g.cB[k] * (qb - qc);
            const T vq = g.dz[k] * qc;
            s0 += vq * rc;
            s1 += vq * aq;
        }
    }
    double x[2] = {(double)s0, (double)s1};
    if (grid_sum<2>(x, red)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            const double a = x[0] / x[1];
            *alpha = (x[1] != 0.0 && isfinite(a)) ? a : 0.0;
            if (in_loop) {
                // the update goes into the SOR correction: hand its "correction
                // is zero" state to k_warm_apply_dl and mark it live for the sweeps
                red.sc->zcopy = red.sc->zflag;
                red.sc->zflag = 0;
            }
        }
    }
}

// The line search with the network's prolongation folded in.  The CTA's
// 32 x 8 x kEstChunk tile and its one-cell halo of q are formed in shared
// memory from the coarse output yc (stride S) with the arithmetic of the
// stand-alone prolongation kernel: the (y, z)-interpolated coarse columns
// once per (plane, row) of the halo box, then each cell's x-interpolation.
// The unknown mask is applied where the value is used: an owned cell takes q
// only if it is an unknown, and a neighbour is read only across an open
// face, which joins two fluid cells that both have an open face, i.e. two
// unknowns, so the halo needs no flags.  Halo cells across a periodic face
// take the wrapped cell's value; other cells outside the grid hold 0 (their
// faces are closed).
// The sums are those of k_warm_ls, in the same order, and the owned cells'
// q goes to qout for the step kernels.
//
// Column slots: the unwrapped halo cells fx in [fa, fb] (at most 34) need the
// coarse columns c0(fa) .. c0(fb) + 1; c0 is floor((f + 1/2)/S - 1/2) before
// the clamp, so c0(fb) - c0(fa) <= floor(33 / S) + 1 and at most
// floor(33 / S) + 3 <= 34 / S + 3 slots are used.  Wrapped cells (a periodic
// x face) take their columns from yc directly.
template <int S>
struct LsTile {
    static constexpr int HX = 34, HY = 10, HZ = kEstChunk + 2, CW = 34 / S + 3;
    float q[HZ][HY][HX];
    float col[HZ][HY][CW];
    float wx[HX], wy[HY], wz[HZ];
    int fx[HX], fy[HY], fz[HZ];          // fine coordinate (wrapped), -1 outside the grid
    int x0[HX], x1[HX];                  // column slots (>= 0) or -1 - coarse column (wrapped cell)
    int y0[HY], y1[HY], z0[HZ], z1[HZ];  // coarse rows and planes
};

// fine coordinate of halo offset f on an axis of n cells: wrapped on a
// periodic axis, else -1 outside the grid
__device__ __forceinline__ int halo_coord(int f, int n, int per) {
    if (f >= 0 && f < n) return f;
    if (!per) return -1;
    f %= n;
    return f < 0 ? f + n : f;
}

template <typename T, int S>
__global__ void __launch_bounds__(256) k_warm_ls_c(Geo<T> g, const T* __restrict__ r, const float* __restrict__ yc,
                                                   float* __restrict__ qout, double* alpha, Reduce red, int in_loop) {
    using LT = LsTile<S>;
    __shared__ LT L;
    // everything up to the dependency wait reads only what no kernel of the
    // solve writes (the geometry and the flags): it overlaps the tail of the
    // convolution before
    const Dom& d = g.d;
    const int tid = threadIdx.x + 32 * threadIdx.y;
    const int Xc = (d.nx + S - 1) / S, Yc = (d.ny + S - 1) / S, Zc = (d.nz + S - 1) / S;
    const int X0 = blockIdx.x * 32 - 1, Y0 = blockIdx.y * 8 - 1, Z0 = blockIdx.z * kEstChunk - 1;
    int cmin;
    {
        float w;
        prolong_w(max(X0, 0), S, Xc, cmin, w);
    }
    // the owned cells' flags, issued first so that their latency overlaps the
    // set-up of the tile (the residuals after the wait)
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = blockIdx.x * 32 + tx + 1, j = blockIdx.y * 8 + ty + 1;
    const int kb = blockIdx.z * kEstChunk + 1, ke = min(kb + kEstChunk, d.nz + 1);
    const bool own = i <= d.nx && j <= d.ny;
    const int pl = (int)d.plane;
    const long long cown = own ? d.at(i, j, kb) : 0;
    uint8_t fl[kEstChunk];
    T rr[kEstChunk];
#pragma unroll
    for (int m = 0; m < kEstChunk; ++m) fl[m] = own && kb + m < ke ? g.flags[cown + (long long)m * pl] : (uint8_t)0;
    if (tid < LT::HX) {
        const int f = X0 + tid, fw = halo_coord(f, d.nx, d.perx);
        const bool wrapped = fw >= 0 && fw != f;
        int c0 = 0;
        float w = 0.f;
        if (fw >= 0) prolong_w(fw, S, Xc, c0, w);
        const int c1 = min(c0 + 1, Xc - 1);
        L.fx[tid] = fw;
        L.wx[tid] = w;
        L.x0[tid] = wrapped ? -1 - c0 : c0 - cmin;
        L.x1[tid] = wrapped ? -1 - c1 : c1 - cmin;
    } else if (tid >= 64 && tid < 64 + LT::HY) {
        const int h = tid - 64, fw = halo_coord(Y0 + h, d.ny, d.pery);
        int c0 = 0;
        float w = 0.f;
        if (fw >= 0) prolong_w(fw, S, Yc, c0, w);
        L.fy[h] = fw;
        L.wy[h] = w;
        L.y0[h] = c0;
        L.y1[h] = min(c0 + 1, Yc - 1);
    } else if (tid >= 96 && tid < 96 + LT::HZ) {
        const int h = tid - 96, fw = halo_coord(Z0 + h, d.nz, d.perz);
        int c0 = 0;
        float w = 0.f;
        if (fw >= 0) prolong_w(fw, S, Zc, c0, w);
        L.fz[h] = fw;
        L.wz[h] = w;
        L.z0[h] = c0;
        L.z1[h] = min(c0 + 1, Zc - 1);
    }
    pdl_wait();
    if (red.sc->done) return;      // uniform over the grid (no barrier has been passed yet)
#pragma unroll
    for (int m = 0; m < kEstChunk; ++m) rr[m] = own && kb + m < ke ? r[cown + (long long)m * pl] : T(0);
    __syncthreads();
    for (int q = tid; q < LT::HZ * LT::HY * LT::CW; q += 256) {
        const int c = q % LT::CW, hy = (q / LT::CW) % LT::HY, hz = q / (LT::CW * LT::HY);
        const int cc = cmin + c;
        float v = 0.f;
        if (cc < Xc && L.fy[hy] >= 0 && L.fz[hz] >= 0)
            v = prolong_col(yc, Xc, Yc, cc, L.y0[hy], L.y1[hy], L.wy[hy], L.z0[hz], L.z1[hz], L.wz[hz]);
        L.col[hz][hy][c] = v;
    }
    __syncthreads();
    // the fine values of the tile: cell (hx, hy, hz) as the x-interpolation of
    // its two coarse columns; warps take rows (hy, hz) with lanes along x (the
    // x weights and column slots of a lane stay in registers), then the last
    // LT::HX - 32 cells of every row go one per thread
    auto fine = [&](int hx, int hy, int hz, int fx, int a, int b, float wxv) {
        float v = 0.f;
        if (fx >= 0 && L.fy[hy] >= 0 && L.fz[hz] >= 0) {
            float v0, v1;
            if (a >= 0) {
                v0 = L.col[hz][hy][a];
                v1 = L.col[hz][hy][b];
            } else {
                v0 = prolong_col(yc, Xc, Yc, -1 - a, L.y0[hy], L.y1[hy], L.wy[hy], L.z0[hz], L.z1[hz], L.wz[hz]);
                v1 = prolong_col(yc, Xc, Yc, -1 - b, L.y0[hy], L.y1[hy], L.wy[hy], L.z0[hz], L.z1[hz], L.wz[hz]);
            }
            v = prolong_mix(v0, v1, wxv);
        }
        L.q[hz][hy][hx] = v;
    };
    static_assert(LT::HX > 32 && LT::HX - 32 <= 2 && (LT::HX - 32) * LT::HY * LT::HZ <= 256, "one tail pass");
    {
        const int fx = L.fx[tx], a = L.x0[tx], b = L.x1[tx];
        const float wxv = L.wx[tx];
        int hy = ty, hz = 0;                   // row ty, ty + 8, ... of the HZ x HY rows
        for (int rw = ty; rw < LT::HZ * LT::HY; rw += 8) {
            fine(tx, hy, hz, fx, a, b, wxv);
            hy += 8;
            while (hy >= LT::HY) {
                hy -= LT::HY;
                ++hz;
            }
        }
        constexpr int NTAIL = LT::HX - 32;
        if (tid < NTAIL * LT::HY * LT::HZ) {
            const int hx = 32 + tid % NTAIL, rw = tid / NTAIL;
            fine(hx, rw % LT::HY, rw / LT::HY, L.fx[hx], L.x0[hx], L.x1[hx], L.wx[hx]);
        }
    }
    __syncthreads();
    T s0 = T(0), s1 = T(0);
    if (own) {
        const int sz = d.nx * d.ny;
        const int v0 = ((kb - 1) * d.ny + (j - 1)) * d.nx + (i - 1);
#pragma unroll
        for (int m = 0; m < kEstChunk; ++m) {
            if (kb + m >= ke) break;
            const float* qq = &L.q[m + 1][ty + 1][tx + 1];
            const uint8_t f = fl[m];
            qout[v0 + m * sz] = (f & F_UNK) ? qq[0] : 0.f;
            if (!(f & F_UNK)) continue;
            const int k = kb + m;
            const T qc = (T)qq[0], rc = rr[m];
            const T qe = (T)qq[1], qw = (T)qq[-1];
            const T qn = (T)qq[LT::HX], qs = (T)qq[-LT::HX];
            const T qt = (T)qq[LT::HY * LT::HX], qb = (T)qq[-LT::HY * LT::HX];
            T aq = T(0);
            if (f & F_E) aq += g.cx * (qe - qc);
            if (f & F_W) aq += g.cx * (qw - qc);
            if (f & F_N) aq += g.cy * (qn - qc);
            if (f & F_S) aq += g.cy * (qs - qc);
            if (f & F_T) aq += g.cT[k] * (qt - qc);
            if (f & F_B) aq += g.cB[k] * (qb - qc);
            const T vq = g.dz[k] * qc;
            s0 += vq * rc;
            s1 += vq * aq;
        }
    }
    double x[2] = {(double)s0, (double)s1};
    if (grid_sum<2>(x, red)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            const double a = x[0] / x[1];
            *alpha = (x[1] != 0.0 && isfinite(a)) ? a : 0.0;
            if (in_loop) {
                red.sc->zcopy = red.sc->zflag;
                red.sc->zflag = 0;
            }
        }
    }
}

// the steps along q: a (32 x 8) column tile over kEstChunk planes per CTA
// (few CTAs: the launch, not the work, bounds these kernels otherwise)
template <typename T>
__global__ void k_warm_apply(Geo<T> g, double* ph, const float* q, const double* alpha, const Scalars* sc) {
    pdl_wait();
    const Dom& d = g.d;
    if (sc->done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    const int kb = blockIdx.z * kEstChunk + 1, ke = min(kb + kEstChunk, d.nz + 1);
    if (i > d.nx || j > d.ny) return;
    const double a = *alpha;
    long long c = d.at(i, j, kb);
    int v = ((kb - 1) * d.ny + (j - 1)) * d.nx + (i - 1);
    for (int k = kb; k < ke; ++k, c += d.plane, v += d.nx * d.ny)
        if (g.flags[c] & F_UNK) ph[c] += a * (double)q[v];
}

// inside the solve loop: the SOR correction d (field type) takes the step,
// d = (zero ? 0 : d) + alpha q, so the FP64 pressure is only touched by the
// next refinement
template <typename T>
__global__ void k_warm_apply_dl(Geo<T> g, T* dl, const float* q, const double* alpha, const Scalars* sc) {
    pdl_wait();
    const Dom& d = g.d;
    if (sc->done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    const int kb = blockIdx.z * kEstChunk + 1, ke = min(kb + kEstChunk, d.nz + 1);
    if (i > d.nx || j > d.ny) return;
    const T a = (T)*alpha;
    const bool zero = sc->zcopy != 0;
    const long long c0 = d.at(i, j, kb);
    const int v0 = ((kb - 1) * d.ny + (j - 1)) * d.nx + (i - 1), sz = d.nx * d.ny;
    // every load of the chunk first (a plane past the chunk reads its first one)
    uint8_t fl[kEstChunk];
    T dv[kEstChunk];
    float qv[kEstChunk];
#pragma unroll
    for (int m = 0; m < kEstChunk; ++m) {
        const bool in = kb + m < ke;
        const long long c = in ? c0 + (long long)m * d.plane : c0;
        fl[m] = in ? g.flags[c] : (uint8_t)0;
        dv[m] = dl[c];
        qv[m] = q[in ? v0 + m * sz : v0];
    }
#pragma unroll
    for (int m = 0; m < kEstChunk; ++m) {
        if (!(fl[m] & F_UNK)) continue;
        const T base = zero ? T(0) : dv[m];
        dl[c0 + (long long)m * d.plane] = base + a * (T)qv[m];
    }
}

// the overlapped correction's step: d = (zero ? 0 : d) + alpha q as in
// k_warm_apply_dl, and r -= alpha (A q) with A q formed exactly as in the
// line search, so r becomes the residual of the corrected iterate
template <typename T>
__global__ void k_warm_apply_dlr(Geo<T> g, T* dl, T* r, const float* __restrict__ q, const double* alpha,
                                 const Scalars* sc) {
    pdl_wait();
    const Dom& d = g.d;
    if (sc->done || !sc->qpend) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    const int kb = blockIdx.z * kEstChunk + 1, ke = min(kb + kEstChunk, d.nz + 1);
    if (i > d.nx || j > d.ny) return;
    const T a = (T)*alpha;
    const bool zero = sc->zcopy != 0;
    const int sy = d.nx, sz = d.nx * d.ny;
    const int oe = (d.perx && i == d.nx) ? -(d.nx - 1) : 1;
    const int ow = (d.perx && i == 1) ? (d.nx - 1) : -1;
    const int on = (d.pery && j == d.ny) ? -(d.ny - 1) * sy : sy;
    const int os = (d.pery && j == 1) ? (d.ny - 1) * sy : -sy;
    long long c = d.at(i, j, kb);
    int v = ((kb - 1) * d.ny + (j - 1)) * d.nx + (i - 1);
    for (int k = kb; k < ke; ++k, c += d.plane, v += sz) {
        const uint8_t f = g.flags[c];
        if (!(f & F_UNK)) continue;
        const int ot = (d.perz && k == d.nz) ? -(d.nz - 1) * sz : sz;
        const int ob = (d.perz && k == 1) ? (d.nz - 1) * sz : -sz;
        const T qc = (T)q[v];
        const T qe = (f & F_E) ? (T)q[v + oe] : T(0), qw = (f & F_W) ? (T)q[v + ow] : T(0);
        const T qn = (f & F_N) ? (T)q[v + on] : T(0), qs = (f & F_S) ? (T)q[v + os] : T(0);
        const T qt = (f & F_T) ? (T)q[v + ot] : T(0), qb = (f & F_B) ? (T)q[v + ob] : T(0);
        T aq = T(0);
        if (f & F_E) aq += g.cx * (qe - qc);
        if (f & F_W) aq += g.cx * (qw - qc);
        if (f & F_N) aq += g.cy * (qn - qc);
        if (f & F_S) aq += g.cy * (qs - qc);
        if (f & F_T) aq += g.cT[k] * (qt - qc);
        if (f & F_B) aq += g.cB[k] * (qb - qc);
        const T base = zero ? T(0) : dl[c];
        dl[c] = base + a * qc;
        r[c] -= a * aq;
    }
}

template <typename T>
int launch_warm_pending(const Geo<T>& g, T* r, const float* q, T* dl, double* alpha, const Reduce& red,
                        cudaStream_t s) {
    const Dom& d = g.d;
    const dim3 grid((d.nx + 31) / 32, (d.ny + 7) / 8, (d.nz + kEstChunk - 1) / kEstChunk), blk(32, 8);
    launch_pdl(k_warm_ls<T>, grid, blk, 0, s, g, (const T*)r, q, alpha, red, 2);
    launch_pdl(k_warm_apply_dlr<T>, grid, blk, 0, s, g, dl, r, q, (const double*)alpha, (const Scalars*)red.sc);
    return 2;
}

__global__ void k_set_flag(int* flag, int value, const int* gate) {
    if (gate && *(volatile const int*)gate) return;
    *flag = value;
}

int launch_set_flag(int* flag, int value, const int* gate, cudaStream_t s) {
    k_set_flag<<<1, 1, 0, s>>>(flag, value, gate);
    return 1;
}

template <typename T>
int launch_warm(const Geo<T>& g, const T* r, const float* q, double* ph, T* dl, double* alpha, const Reduce& red,
                cudaStream_t s) {
    const Dom& d = g.d;
    const dim3 grid((d.nx + 31) / 32, (d.ny + 7) / 8, (d.nz + kEstChunk - 1) / kEstChunk), blk(32, 8);
    launch_pdl(k_warm_ls<T>, grid, blk, 0, s, g, r, q, alpha, red, dl ? 1 : 0);
    if (dl)
        launch_pdl(k_warm_apply_dl<T>, grid, blk, 0, s, g, dl, q, alpha, (const Scalars*)red.sc);
    else
        launch_pdl(k_warm_apply<T>, grid, blk, 0, s, g, ph, q, alpha, (const Scalars*)red.sc);
    return 2;
}

template <typename T>
int launch_warm_coarse(const Geo<T>& g, const T* r, const float* yc, int st, float* q, double* ph, T* dl,
                       double* alpha, const Reduce& red, cudaStream_t s) {
    const Dom& d = g.d;
    const dim3 grid((d.nx + 31) / 32, (d.ny + 7) / 8, (d.nz + kEstChunk - 1) / kEstChunk), blk(32, 8);
    const int il = dl ? 1 : 0;
    switch (st) {
        case 1: launch_pdl(k_warm_ls_c<T, 1>, grid, blk, 0, s, g, r, yc, q, alpha, red, il); break;
        case 2: launch_pdl(k_warm_ls_c<T, 2>, grid, blk, 0, s, g, r, yc, q, alpha, red, il); break;
        case 4: launch_pdl(k_warm_ls_c<T, 4>, grid, blk, 0, s, g, r, yc, q, alpha, red, il); break;
        default: launch_pdl(k_warm_ls_c<T, 8>, grid, blk, 0, s, g, r, yc, q, alpha, red, il); break;
    }
    if (dl)
        launch_pdl(k_warm_apply_dl<T>, grid, blk, 0, s, g, dl, (const float*)q, (const double*)alpha,
                   (const Scalars*)red.sc);
    else
        launch_pdl(k_warm_apply<T>, grid, blk, 0, s, g, ph, (const float*)q, (const double*)alpha,
                   (const Scalars*)red.sc);
    return 2;
}

// training pairs: delta = ph - ph0 (the correction a solve applied, before the gauge)
template <typename T>
__global__ void k_record_delta(Geo<T> g, const double* ph, const double* ph0, T* out) {
    const Dom& d = g.d;
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    const int k = blockIdx.z + 1;
    if (i > d.nx || j > d.ny) return;
    const long long c = d.at(i, j, k);
    out[c] = (g.flags[c] & F_UNK) ? (T)(ph[c] - ph0[c]) : T(0);
}
template <typename T>
__global__ void k_unknown_mask(Geo<T> g, T* out) {
    const Dom& d = g.d;
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    const int k = blockIdx.z + 1;
    if (i > d.nx || j > d.ny) return;
    const long long c = d.at(i, j, k);
    out[c] = (g.flags[c] & F_UNK) ? T(1) : T(0);
}
template <typename T>
int launch_record(const Geo<T>& g, const double* ph, const double* ph0, T* out, int what, cudaStream_t s) {
    const Dom& d = g.d;
    const dim3 grid((d.nx + 31) / 32, (d.ny + 7) / 8, d.nz), blk(32, 8);
    if (what == 0) k_record_delta<T><<<grid, blk, 0, s>>>(g, ph, ph0, out);
    else k_unknown_mask<T><<<grid, blk, 0, s>>>(g, out);
    return 1;
}

__global__ void k_count_unknowns(Dom d, const uint8_t* flags, unsigned long long* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    const int k = blockIdx.z + 1;
    unsigned v = 0;
    if (i <= d.nx && j <= d.ny) v = (flags[d.at(i, j, k)] & F_UNK) ? 1u : 0u;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (((threadIdx.x + threadIdx.y * blockDim.x) & 31) == 0 && v) atomicAdd(out, (unsigned long long)v);
}
int launch_count_unknowns(const Dom& d, const uint8_t* flags, unsigned long long* out, cudaStream_t s) {
    k_count_unknowns<<<dim3((d.nx + 31) / 32, (d.ny + 7) / 8, d.nz), dim3(32, 8), 0, s>>>(d, flags, out);
    return 1;
}

// ---------------------------------------------------------------------------
// Comparison of SOR variants (les_sor_compare): the FP64 residual of a given
// pressure without the solver's bookkeeping, p0 + d, and the paper's twinned
// double-buffer half-sweep (Sec. 2.6).

// r = b - A p (FP64, stored in T) on the unknowns, 0 elsewhere; out[0] =
// ||r||^2, out[1] = ||b||^2 over the unknowns (last-block sums)
template <typename T>
__global__ void __launch_bounds__(256) k_cmp_residual(Geo<T> g, const double* p, const double* b, T* r, Reduce red,
                                                      double* out) {
    const Dom& d = g.d;
    const int n = d.nx * d.ny * d.nz;
    double x[2] = {0.0, 0.0};
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        int i, j, k;
        cell_of(d, q, i, j, k);
        const long long c = d.at(i, j, k);
        const uint8_t f = g.flags[c];
        if (!(f & F_UNK)) {
            r[c] = T(0);
            continue;
        }
        Poisson<T> Q{g};
        double ae, aw, an, as, at, ab;
        Q.coefs(f, k, g.cx64, g.cy64, g.cT64, g.cB64, ae, aw, an, as, at, ab);
        long long e, w, nn, s_, t, bt;
        Q.nbr(i, j, k, e, w, nn, s_, t, bt);
        double s = 0.0;
        s += ae * p[e];
        s += aw * p[w];
        s += an * p[nn];
        s += as * p[s_];
        s += at * p[t];
        s += ab * p[bt];
        const double res = b[c] - (s - g.diag64[k * 64 + (f & 63)] * p[c]);
        r[c] = (T)res;
        x[0] += res * res;
        x[1] += b[c] * b[c];
    }
    if (grid_sum_at<2>(x, red, gridDim.x, blockIdx.x)) {
        if (threadIdx.x == 0) {
            out[0] = x[0];
            out[1] = x[1];
        }
    }
}

template <typename T>
int launch_cmp_residual(const Geo<T>& g, const double* p, const double* b, T* r, const Reduce& red, double* out,
                        cudaStream_t s) {
    k_cmp_residual<T><<<reduce_blocks(g.d), 256, 0, s>>>(g, p, b, r, red, out);
    return 1;
}

// p_new = p0 + d on the unknowns (d read with a stride: 2 for one copy of a
// twinned pair array), p0 elsewhere; over the whole padded array
template <typename T>
__global__ void k_cmp_add(const uint8_t* flags, const double* p0, const T* dv, int stride, double* pn, size_t n) {
    const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    pn[c] = p0[c] + ((flags[c] & F_UNK) ? (double)dv[c * stride] : 0.0);
}

template <typename T>
int launch_cmp_add(const Geo<T>& g, const double* p0, const T* dv, int stride, double* pn, size_t n,
                   cudaStream_t s) {
    k_cmp_add<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g.flags, p0, dv, stride, pn, n);
    return 1;
}

// the two copies of a twinned correction, interleaved (the paper's array of
// two-element vectors): one aligned access reads both
template <typename T>
struct alignas(2 * sizeof(T)) Twin {
    T c[2];
};

// One half of a twinned double-buffer sweep (Sec. 2.6) on the correction
// equation A d = r: copy 1 - nrd of every unknown takes the printed update
// with its own value and every neighbour from copy nrd (the same per-cell
// arithmetic as the red-black kernels).  A 32 x 8 column tile walks kc planes.
template <typename T>
__global__ void k_twin_half(Geo<T> g, Twin<T>* tw, const T* __restrict__ r, int nrd, T omega, int kc) {
    const Dom& d = g.d;
    const int i = blockIdx.x * 32 + threadIdx.x + 1, j = blockIdx.y * 8 + threadIdx.y + 1;
    const int kb = blockIdx.z * kc + 1, ke = min(kb + kc, d.nz + 1);
    if (i > d.nx || j > d.ny) return;
    const int src = nrd, dst = 1 - nrd;
    const int pl = (int)d.plane;
    const int oe = (d.perx && i == d.nx) ? -(d.nx - 1) : 1;
    const int ow = (d.perx && i == 1) ? (d.nx - 1) : -1;
    const int on = (d.pery && j == d.ny) ? -(d.ny - 1) * d.px : d.px;
    const int os = (d.pery && j == 1) ? (d.ny - 1) * d.px : -d.px;
    long long c = d.at(i, j, kb);
    for (int k = kb; k < ke; ++k, c += pl) {
        const uint8_t f = g.flags[c];
        if (!(f & F_UNK)) continue;
        const int ot = (d.perz && k == d.nz) ? -(d.nz - 1) * pl : pl;
        const int ob = (d.perz && k == 1) ? (d.nz - 1) * pl : -pl;
        const T ae = (f & F_E) ? g.cx : T(0), aw = (f & F_W) ? g.cx : T(0);
        const T an = (f & F_N) ? g.cy : T(0), as = (f & F_S) ? g.cy : T(0);
        const T at = (f & F_T) ? g.cT[k] : T(0), ab = (f & F_B) ? g.cB[k] : T(0);
        const T cn1 = T(1) / (ae + aw + an + as + at + ab);
        const Twin<T> ve = tw[c + oe], vw = tw[c + ow], vn = tw[c + on], vs = tw[c + os], vt = tw[c + ot],
                      vb = tw[c + ob], vc = tw[c];
        T s = T(0);
        s += ae * ve.c[src];
        s += aw * vw.c[src];
        s += an * vn.c[src];
        s += as * vs.c[src];
        s += at * vt.c[src];
        s += ab * vb.c[src];
        const T own = vc.c[src];
        const T reltmp = omega * (cn1 * (s - r[c]) - own);
        tw[c].c[dst] = own + reltmp;
    }
}

template <typename T>
int launch_twin_half(const Geo<T>& g, void* tw, const T* r, int nrd, T omega, cudaStream_t s) {
    const Dom& d = g.d;
    const int kc = accum_kc(d);
    k_twin_half<T><<<dim3((d.nx + 31) / 32, (d.ny + 7) / 8, (d.nz + kc - 1) / kc), dim3(32, 8), 0, s>>>(
        g, (Twin<T>*)tw, r, nrd, omega, kc);
    return 1;
}

// FP64 diagonal of the Poisson operator over (plane, open-face mask): the
// sum of the open faces' coefficients in the order of the residual kernels
template <typename T>
__global__ void k_diag_table(Geo<T> g, double* tab) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (g.d.nz + 2) * 64) return;
    const int k = q >> 6, m = q & 63;
    Poisson<T> Q{g};
    double ae, aw, an, as, at, ab;
    Q.coefs((uint8_t)m, k, g.cx64, g.cy64, g.cT64, g.cB64, ae, aw, an, as, at, ab);
    tab[q] = ae + aw + an + as + at + ab;
}

template <typename T>
int launch_diag_table(const Geo<T>& g, double* tab, cudaStream_t s) {
    const int n = (g.d.nz + 2) * 64;
    k_diag_table<T><<<(n + 255) / 256, 256, 0, s>>>(g, tab);
    return 1;
}

int max_reduce_blocks(const Dom& d) { return ((d.nx + 31) / 32) * ((d.ny + 7) / 8) * d.nz; }

// ---------------------------------------------------------------------------
// ensembles: the estimate and the refinement of every member in one launch
// each, block by block the same geometry as the member's own launch (so the
// sums, the decisions and the iterates are bit-identical)

__device__ __forceinline__ int ens_member(const int* beg, int n, int t) {
    int m = 0;
    while (m + 1 < n && t >= beg[m + 1]) ++m;
    return m;
}

__global__ void __launch_bounds__(256, 4) k_sor_est_ens(const __grid_constant__ EnsTab<float> tab, int dcur,
                                                        CondArgs ca) {
    const int t = blockIdx.x, m = ens_member(tab.ebeg, tab.n, t);
    const EnsMember<float>& M = tab.m[m];
    if (M.red.sc->done) return;
    CondArgs c = ca;
    c.tol = M.tol;
    c.limit = M.limit;
    const int lt = t - tab.ebeg[m], ex = M.egrid[0], ey = M.egrid[1];
    sor_est_body<float>(M.g, M.dl[dcur], M.rr, M.rcur, M.red, c, lt % ex, (lt / ex) % ey, lt / (ex * ey),
                        ex * ey * M.egrid[2], lt);
}

__global__ void k_accum_ens(const __grid_constant__ EnsTab<float> tab, int dcur) {
    const int t = blockIdx.x, m = ens_member(tab.abeg, tab.n, t);
    const EnsMember<float>& M = tab.m[m];
    if (M.red.sc->done || !M.red.sc->refine) return;
    const int lt = t - tab.abeg[m], ax = M.agrid[0], ay = M.agrid[1];
    accum_body<float>(M.g, M.ph, M.dl[dcur], lt % ax, (lt / ax) % ay, lt / (ax * ay));
}

__global__ void __launch_bounds__(256) k_residual64_ens(const __grid_constant__ EnsTab<float> tab, CondArgs ca) {
    const int t = blockIdx.x, m = ens_member(tab.rbeg, tab.n, t);
    const EnsMember<float>& M = tab.m[m];
    if (ca.gate == 1 && (M.red.sc->done || !M.red.sc->refine)) return;
    if (ca.gate == 2 && M.red.sc->done) return;
    CondArgs c = ca;
    c.tol = M.tol;
    c.limit = M.limit;
    c.done_host = nullptr;
    const int done = residual64_body<float>(M.g, M.ph, M.rhs, M.rr, M.vfluid, M.red, c, t - tab.rbeg[m],
                                            M.rblocks);
    if (done == 1 && tab.ndone) {
        // this member's solve ended: the last member to end raises the host flag
        const int v = atomicAdd(tab.ndone, 1) + 1;
        if (v == tab.n && tab.all_done_host) *(volatile int*)tab.all_done_host = 1;
    }
}

// ---------------------------------------------------------------------------
// The plain-SOR solve of an ensemble in one persistent cooperative launch:
// every CTA walks, batch after batch, the flattened items of each phase --
// `cycle` sweeps over every running member's 28 x 8 x 8 TMA blocks (with the
// member's tensor maps), the estimate, the gated FP64 accumulation and the
// gated FP64 residual with its stop decision -- the same per-item bodies as
// the batched launches, separated by a bounded grid barrier, until every
// member's solve has ended.  Members that have stopped are skipped.  The
// launch count of a step no longer depends on its sweeps.

// bounded grid barrier (1 s of global time); false on a timeout (recorded)
__device__ bool ens_grid_barrier(unsigned* bar, int* err) {
    __shared__ int ok_sh;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    __syncthreads();
    if (tid == 0) {
        unsigned* count = bar;
        unsigned* gen = bar + 1;
        const unsigned g0 = *(volatile unsigned*)gen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(count, 1u) == gridDim.x - 1) {
            *(volatile unsigned*)count = 0u;
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const uint64_t t0 = tma::global_ns();
            while (*(volatile unsigned*)gen == g0)
                if (tma::global_ns() - t0 > 1000000000ull) {
                    ok = 0;
                    atomicExch(err, 1);
                    break;
                }
        }
        __threadfence();
        ok_sh = ok && !*(volatile int*)err;
    }
    __syncthreads();
    return ok_sh != 0;
}

__global__ void __launch_bounds__(256) k_ens_persist(const __grid_constant__ EnsTab<float> tab,
                                                     const CUtensorMap* __restrict__ maps, int cycle, int batches,
                                                     CondArgs ca, unsigned* bar, int* err) {
    using TT = tma::TmaTile<kEnsTmaBy, kEnsTmaBz>;
    extern __shared__ __align__(128) unsigned char psm[];
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int n = tab.n;
    if (tid == 0) {
        tma::mbar_init(tma::smem_u32(psm + tma::ColTile<kEnsTmaBy, kEnsTmaBz>::STAGE), 1);
        tma::mbar_fence_init();
    }
    // the maps were written through the generic proxy (a host copy): acquire
    // them for the tensor-map proxy once per CTA, one map per thread
    for (int c = tid; c < 4 * n; c += 256)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(maps + c) : "memory");
    __syncthreads();
    uint32_t phase = 0;
    for (int b = 0; b < batches; ++b) {
        for (int s = 0; s < cycle; ++s) {
            const int in = s & 1;
            int m = 0;
            for (int t = blockIdx.x; t < tab.tbeg[n]; t += gridDim.x) {
                while (t >= tab.tbeg[m + 1]) ++m;
                const EnsMember<float>& M = tab.m[m];
                Scalars* sc = M.red.sc;
                if (*(volatile const int*)&sc->done) continue;
                const Dom& d = M.g.d;
                const int gx = (d.nx + TT::BX - 1) / TT::BX, gy = (d.ny + kEnsTmaBy - 1) / kEnsTmaBy;
                const int q = t - tab.tbeg[m];
                const bool zero_start = s == 0 && sc->zflag;
                const CUtensorMap* mm = maps + 4 * m;
                if (!tma::sor_col_block<kEnsTmaBy, kEnsTmaBz, 256>(psm, mm + in, mm + 2, mm + 3, M.g, M.dl[in], M.rr,
                                                                    M.dl[1 - in], zero_start, sc, q % gx,
                                                                    (q / gx) % gy, q / (gx * gy), phase)) {
                    if (tid == 0) atomicExch(err, 1);
                    break;
                }
                phase ^= 1u;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncthreads();
            }
            if (!ens_grid_barrier(bar, err)) return;
        }
        {   // estimate of every running member
            int m = 0;
            for (int t = blockIdx.x; t < tab.ebeg[n]; t += gridDim.x) {
                while (t >= tab.ebeg[m + 1]) ++m;
                const EnsMember<float>& M = tab.m[m];
                if (M.red.sc->done) continue;
                CondArgs c = ca;
                c.tol = M.tol;
                c.limit = M.limit;
                const int lt = t - tab.ebeg[m], ex = M.egrid[0], ey = M.egrid[1];
                sor_est_body<float>(M.g, M.dl[0], M.rr, M.rcur, M.red, c, lt % ex, (lt / ex) % ey, lt / (ex * ey),
                                    ex * ey * M.egrid[2], lt);
            }
        }
        if (!ens_grid_barrier(bar, err)) return;
        {   // FP64 accumulation where a refinement was asked for
            int m = 0;
            for (int t = blockIdx.x; t < tab.abeg[n]; t += gridDim.x) {
                while (t >= tab.abeg[m + 1]) ++m;
                const EnsMember<float>& M = tab.m[m];
                if (M.red.sc->done || !M.red.sc->refine) continue;
                const int lt = t - tab.abeg[m], ax = M.agrid[0], ay = M.agrid[1];
                accum_body<float>(M.g, M.ph, M.dl[0], lt % ax, (lt / ax) % ay, lt / (ax * ay));
            }
        }
        if (!ens_grid_barrier(bar, err)) return;
        {   // FP64 residual and stop decision
            int m = 0;
            for (int t = blockIdx.x; t < tab.rbeg[n]; t += gridDim.x) {
                while (t >= tab.rbeg[m + 1]) ++m;
                const EnsMember<float>& M = tab.m[m];
                if (M.red.sc->done || !M.red.sc->refine) continue;
                CondArgs c = ca;
                c.tol = M.tol;
                c.limit = M.limit;
                c.done_host = nullptr;
                const int done = residual64_body<float>(M.g, M.ph, M.rhs, M.rr, M.vfluid, M.red, c,
                                                        t - tab.rbeg[m], M.rblocks);
                if (done == 1 && tab.ndone) {
                    const int v = atomicAdd(tab.ndone, 1) + 1;
                    if (v == n && tab.all_done_host) *(volatile int*)tab.all_done_host = 1;
                }
            }
        }
        if (!ens_grid_barrier(bar, err)) return;
        if (*(volatile int*)tab.ndone >= n) break;      // every member's solve has ended
    }
}

int ens_persist_grid() {
    static int grid = -1;
    if (grid < 0) {
        using TT = tma::ColTile<kEnsTmaBy, kEnsTmaBz>;
        int dev = 0, sms = 0, per = 0, coop = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        if (cudaFuncSetAttribute(k_ens_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TT::SMEM) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ens_persist, 256, TT::SMEM) != cudaSuccess)
            per = 0;
        grid = coop ? sms * per : 0;
        cudaGetLastError();
    }
    return grid;
}

int launch_ens_persist(const EnsTab<float>& tab, const CUtensorMap* maps, int cycle, int batches, const CondArgs& ca,
                       unsigned* bar, int* err, cudaStream_t s) {
    const int grid = ens_persist_grid();
    if (grid <= 0) return -1;
    using TT = tma::ColTile<kEnsTmaBy, kEnsTmaBz>;
    EnsTab<float> T = tab;
    void* args[] = {(void*)&T, (void*)&maps, (void*)&cycle, (void*)&batches, (void*)&ca, (void*)&bar, (void*)&err};
    if (cudaLaunchCooperativeKernel((const void*)k_ens_persist, dim3(grid), dim3(32, 8), args, TT::SMEM, s) !=
        cudaSuccess)
        return -1;
    return 1;
}

int launch_est_ens(const EnsTab<float>& tab, int dcur, const CondArgs& ca, cudaStream_t s) {
    k_sor_est_ens<<<tab.ebeg[tab.n], dim3(32, 8), 0, s>>>(tab, dcur, ca);
    return 1;
}

int launch_refine_ens(const EnsTab<float>& tab, int dcur, const CondArgs& ca, cudaStream_t s) {
    if (ca.mode != RES_INIT) k_accum_ens<<<tab.abeg[tab.n], dim3(32, 8), 0, s>>>(tab, dcur);
    k_residual64_ens<<<tab.rbeg[tab.n], 256, 0, s>>>(tab, ca);
    return ca.mode != RES_INIT ? 2 : 1;
}

#define LES_INSTANTIATE(T)                                                                              \
    template int launch_bc<T>(const Geo<T>&, T*, T*, T*, const double*, const InflowSeries&, double,      \
                              uint64_t, const Scalars*, cudaStream_t);                                  \
    template int launch_nut<T>(const Geo<T>&, const T*, const T*, const T*, T*, cudaStream_t);          \
    template int launch_momentum<T>(const Geo<T>&, const T*, const T*, const T*, const T*, T*, T*, T*,  \
                                    T*, T*, T*, const Scalars*, cudaStream_t);                          \
    template int launch_outflow<T>(const Geo<T>&, const T*, T*, T*, T*, const Reduce&, cudaStream_t);   \
    template int launch_rhs<T>(const Geo<T>&, const T*, const T*, const T*, T*, double, const Reduce&,  \
                               cudaStream_t);                                                           \
    template int launch_rhs_mean<T>(const Geo<T>&, T*, double, const Reduce&, cudaStream_t);            \
    template int launch_sor_sweep<T>(const Geo<T>&, T*, const T*, int, const Scalars*, cudaStream_t);   \
    template int launch_accum<T>(const Geo<T>&, double*, const T*, const Scalars*, int, cudaStream_t);  \
    template int launch_residual64<T>(const Geo<T>&, const double*, const T*, T*, double, const Reduce&, \
                                      CondArgs, cudaStream_t);                                          \
    template int launch_sor_est<T>(const Geo<T>&, const T*, const T*, T*, const Reduce&, CondArgs, cudaStream_t); \
    template int launch_project<T>(const Geo<T>&, const T*, const T*, const T*, T*, T*, T*,             \
                                   const double*, double*, Scalars*, cudaStream_t);                     \
    template int launch_rhs_eff<T>(const Geo<T>&, const T*, T*, const Scalars*, cudaStream_t);          \
    template int launch_diag_table<T>(const Geo<T>&, double*, cudaStream_t);                          \
    template int launch_cmp_residual<T>(const Geo<T>&, const double*, const double*, T*, const Reduce&,       \
                                        double*, cudaStream_t);                                          \
    template int launch_cmp_add<T>(const Geo<T>&, const double*, const T*, int, double*, size_t,            \
                                   cudaStream_t);                                                       \
    template int launch_twin_half<T>(const Geo<T>&, void*, const T*, int, T, cudaStream_t);               \
    template int launch_gauge<T>(const Geo<T>&, const double*, double*, const Scalars*, cudaStream_t);   \
    template int launch_warm<T>(const Geo<T>&, const T*, const float*, double*, T*, double*, const Reduce&,     \
                                cudaStream_t);                                                          \
    template int launch_warm_pending<T>(const Geo<T>&, T*, const float*, T*, double*, const Reduce&,            \
                                        cudaStream_t);                                                  \
    template int launch_warm_coarse<T>(const Geo<T>&, const T*, const float*, int, float*, double*, T*, double*, \
                                       const Reduce&, cudaStream_t);                                    \
    template int launch_record<T>(const Geo<T>&, const double*, const double*, T*, int, cudaStream_t);

LES_INSTANTIATE(float)
LES_INSTANTIATE(double)

}  // namespace les
