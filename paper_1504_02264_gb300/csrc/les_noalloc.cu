// Poisson residual norms without any device allocation.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// framework's memory pool or arena, applications that must not grow the
// device heap after start-up (a fixed memory budget decided at launch), and
// callers that issue work while a CUDA graph is being captured elsewhere.
// les_residual_noalloc serves them: the caller passes its own device buffers
// for inputs and outputs, and the only scratch this routine needs (one FP64
// partial sum pair per thread block and a completion counter) lives in the
// fixed file-scope device array below.  Nothing here calls cudaMalloc,
// cudaFree or any allocating library routine.
//
// The fixed array is placed on a device when the library's module is loaded
// there.  With CUDA's default lazy module loading that happens at the first
// les_residual_noalloc call on the device (inside cudaGetSymbolAddress), so
// that first call is the one that can grow device memory: fixed-budget
// callers make it at start-up (or set CUDA_MODULE_LOADING=EAGER, which loads
// the module with the context).  From then on the array (about 64 KB) stays
// resident on that GPU until the process exits.
#include <mutex>

#include "../../include/les.h"
#include "les_internal.cuh"

namespace les {
namespace {

constexpr int kNaBlocks = 4096;       // partial-sum slots: at most this many thread blocks
constexpr int kNaThreads = 256;
constexpr int kNaMaxDevices = 64;

// [0]: completion counter (as unsigned), [1 .. 2*kNaBlocks]: partial sums
static __device__ __align__(256) double g_na_scratch[1 + 2 * kNaBlocks];

// per device: the array's address and the context it was looked up in (a
// device reset or a released primary context loads the module again, maybe
// elsewhere; a different current context means the address is looked up again)
void* g_na_ptr[kNaMaxDevices] = {};
CUcontext g_na_ctx[kNaMaxDevices] = {};
std::mutex g_na_mutex;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);

CUcontext current_context() {
    static CtxGetCurrentFn fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        fn = (CtxGetCurrentFn)f;
    }
    CUcontext c = nullptr;
    return fn(&c) == CUDA_SUCCESS ? c : nullptr;
}

__device__ __forceinline__ bool na_fluid(const uint8_t* solid, const Dom& d, int i, int j, int k) {
    if (d.perx) i = i < 0 ? i + d.nx : (i >= d.nx ? i - d.nx : i);
    if (d.pery) j = j < 0 ? j + d.ny : (j >= d.ny ? j - d.ny : j);
    if (d.perz) k = k < 0 ? k + d.nz : (k >= d.nz ? k - d.nz : k);
    if (i < 0 || i >= d.nx || j < 0 || j >= d.ny || k < 0 || k >= d.nz) return false;
    return solid[((long long)k * d.ny + j) * d.nx + i] == 0;
}

// Same residual as the handle path's k_residual64: on every fluid cell with
// an open face, r = rhs - sum_nb a_nb (p_nb - p_c) with the coefficients of
// the printed SOR (open-face indicators times 1/dx^2, 1/dy^2,
// 1/(dz_k dzs_k), 1/(dz_k dzs_{k-1})), accumulated in FP64.  Dense (nz, ny,
// nx) arrays, 0-based indices.
template <typename T>
__global__ void __launch_bounds__(kNaThreads)
k_residual_noalloc(Dom d, double dx, double dy, const T* p, const T* rhs, const uint8_t* solid, const double* dz,
                   double* out, double* scratch) {
    const long long n = (long long)d.nx * d.ny * d.nz;
    const double cx = 1.0 / (dx * dx), cy = 1.0 / (dy * dy);
    double x[2] = {0.0, 0.0};
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % d.nx);
        const long long t = q / d.nx;
        const int j = (int)(t % d.ny);
        const int k = (int)(t / d.ny);
        if (!na_fluid(solid, d, i, j, k)) continue;
        auto dzk = [&](int kk) -> double {   // ghost spacing: mirror, or wrap when periodic
            if (kk < 0) return d.perz ? dz[d.nz - 1] : dz[0];
            if (kk >= d.nz) return d.perz ? dz[0] : dz[d.nz - 1];
            return dz[kk];
        };
        const double dzc = dz[k];
        const double dzs_t = 0.5 * (dzc + dzk(k + 1)), dzs_b = 0.5 * (dzk(k - 1) + dzc);
        const bool bx = !d.perx, by = !d.pery, bz = !d.perz;
        const bool oe = !(bx && i == d.nx - 1) && na_fluid(solid, d, i + 1, j, k);
        const bool ow = !(bx && i == 0) && na_fluid(solid, d, i - 1, j, k);
        const bool on = !(by && j == d.ny - 1) && na_fluid(solid, d, i, j + 1, k);
        const bool os = !(by && j == 0) && na_fluid(solid, d, i, j - 1, k);
        const bool ot = !(bz && k == d.nz - 1) && na_fluid(solid, d, i, j, k + 1);
        const bool ob = !(bz && k == 0) && na_fluid(solid, d, i, j, k - 1);
        if (!(oe || ow || on || os || ot || ob)) continue;
        auto P = [&](int a, int b, int c) -> double {
            if (d.perx) a = a < 0 ? a + d.nx : (a >= d.nx ? a - d.nx : a);
            if (d.pery) b = b < 0 ? b + d.ny : (b >= d.ny ? b - d.ny : b);
            if (d.perz) c = c < 0 ? c + d.nz : (c >= d.nz ? c - d.nz : c);
            return (double)p[((long long)c * d.ny + b) * d.nx + a];
        };
        const double ae = oe ? cx : 0.0, aw = ow ? cx : 0.0, an = on ? cy : 0.0, as = os ? cy : 0.0;
        const double at = ot ? 1.0 / (dzc * dzs_t) : 0.0, ab = ob ? 1.0 / (dzc * dzs_b) : 0.0;
        double s = 0.0;
        if (oe) s += ae * P(i + 1, j, k);
        if (ow) s += aw * P(i - 1, j, k);
        if (on) s += an * P(i, j + 1, k);
        if (os) s += as * P(i, j - 1, k);
        if (ot) s += at * P(i, j, k + 1);
        if (ob) s += ab * P(i, j, k - 1);
        const double diag = ae + aw + an + as + at + ab;
        const double b = (double)rhs[q];
        const double r = b - (s - diag * (double)p[q]);
        x[0] += r * r;
        x[1] += b * b;
    }
    // block sum (warp shuffles, then one value per warp)
    __shared__ double sh[2][kNaThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int v = 0; v < 2; ++v)
        for (int o = 16; o > 0; o >>= 1) x[v] += __shfl_down_sync(0xffffffffu, x[v], o);
    if (lane == 0) {
        sh[0][warp] = x[0];
        sh[1][warp] = x[1];
    }
    __syncthreads();
    unsigned* counter = reinterpret_cast<unsigned*>(scratch);
    double* part = scratch + 1;
    __shared__ bool last;
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kNaThreads / 32; ++w) {
            a += sh[0][w];
            b += sh[1][w];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) {     // fixed order: the result does not depend on block timing
        double a = 0.0, b = 0.0;
        for (unsigned m = 0; m < gridDim.x; ++m) {
            a += __ldcg(&part[2 * m]);
            b += __ldcg(&part[2 * m + 1]);
        }
        out[0] = a;
        out[1] = b;
        out[2] = b == 0.0 ? sqrt(a) : sqrt(a / b);
        *counter = 0u;
    }
}

}  // namespace
}  // namespace les

using namespace les;

extern "C" int les_residual_noalloc(const les_grid_t* grid, const void* d_p, const void* d_rhs,
                                    const uint8_t* d_solid, const double* d_dz, double* d_out, void* stream) {
    if (!grid || !d_p || !d_rhs || !d_solid || !d_dz || !d_out) return LES_EINVAL;
    if (grid->nx < 2 || grid->ny < 2 || grid->nz < 2) return LES_EINVAL;
    const long long n = (long long)grid->nx * grid->ny * grid->nz;
    if (n > (long long)LES_NOALLOC_MAX_CELLS) return LES_EINVAL;
    if (grid->precision != LES_FP32 && grid->precision != LES_FP64) return LES_EINVAL;
    if (!(grid->dx > 0) || !(grid->dy > 0)) return LES_EINVAL;
    if (grid->bc_x != LES_BC_INOUT && grid->bc_x != LES_BC_PERIODIC) return LES_EINVAL;
    if (grid->bc_y != LES_BC_FREESLIP && grid->bc_y != LES_BC_PERIODIC) return LES_EINVAL;
    if (grid->bc_z != LES_BC_WALL && grid->bc_z != LES_BC_PERIODIC) return LES_EINVAL;

    // once per device (and again if the device's context changed), with that
    // device current: the device address of the fixed scratch array (its
    // host-side name is only a stand-in)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return LES_ECUDA;
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ptr[dev] || current_context() != g_na_ctx[dev]) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_na_scratch) != cudaSuccess || !ptr) return LES_ECUDA;
            g_na_ptr[dev] = ptr;
            g_na_ctx[dev] = current_context();        // the lookup made the device's context current
        }
        scratch = g_na_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the counter must start at zero even if an earlier call was interrupted
    if (cudaMemsetAsync(scratch, 0, sizeof(double), s) != cudaSuccess) return LES_ECUDA;

    Dom d{};
    d.nx = grid->nx;
    d.ny = grid->ny;
    d.nz = grid->nz;
    d.perx = grid->bc_x == LES_BC_PERIODIC;
    d.pery = grid->bc_y == LES_BC_PERIODIC;
    d.perz = grid->bc_z == LES_BC_PERIODIC;
    long long nb = (n + kNaThreads - 1) / kNaThreads;
    const unsigned blocks = (unsigned)(nb < kNaBlocks ? nb : kNaBlocks);
    if (grid->precision == LES_FP64)
        k_residual_noalloc<double><<<blocks, kNaThreads, 0, s>>>(d, grid->dx, grid->dy, (const double*)d_p,
                                                                 (const double*)d_rhs, d_solid, d_dz, d_out,
                                                                 (double*)scratch);
    else
        k_residual_noalloc<float><<<blocks, kNaThreads, 0, s>>>(d, grid->dx, grid->dy, (const float*)d_p,
                                                                (const float*)d_rhs, d_solid, d_dz, d_out,
                                                                (double*)scratch);
    return cudaGetLastError() == cudaSuccess ? LES_OK : LES_ECUDA;
}
