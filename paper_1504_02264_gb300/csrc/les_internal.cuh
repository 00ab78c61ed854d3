// Internal declarations of the LES CUDA library (not part of the C ABI).
//
// Device layout: every field is one padded 3-D array of (nz+2) planes of
// (ny+2) rows of `px` elements, i fastest.  Index 0 and n+1 are the ghost
// layer on each axis (1-based interior like the paper's Fortran).  Column
// OX + i holds index i, so the first interior element (i = 1) of every row
// sits on a 16-byte boundary for vector loads; px is a multiple of 16
// elements so every row starts 64-byte aligned.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/les.h"

#include <utility>

namespace les {

// Programmatic dependent launch.  A kernel launched with launch_pdl may be
// scheduled while the previous kernel of its stream is still finishing; its
// first statement, pdl_wait(), blocks until that kernel has completed and its
// writes are visible, so no read or write of the kernel can overlap it.  For
// an ordinary launch pdl_wait() returns at once.  (No kernel triggers its
// dependents early: with griddepcontrol.launch_dependents after the wait,
// the SOR sweeps measured 2% slower on GB300 and the learned step 1%.)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

constexpr int OX = 3;

// Trilinear prolongation of a cell-centred coarse field of stride s to the
// fine cells: fine centre f sits at coarse coordinate (f + 1/2)/s - 1/2 on
// each axis, clamped to the first / last coarse centre; a fine value is the
// x-interpolation of the two (y, z)-interpolated coarse columns around it.
// Shared by the network's prolongation kernel and the line search that
// prolongs on the fly.  Every operation is an explicitly rounded intrinsic,
// so the compiler cannot contract the two kernels' copies differently and
// both form bit-identical values.
__device__ __forceinline__ void prolong_w(int f, int s, int C, int& c0, float& w) {
    const float x = __fsub_rn(__fdiv_rn(__fadd_rn((float)f, 0.5f), (float)s), 0.5f);
    c0 = (int)floorf(x);
    w = __fsub_rn(x, (float)c0);
    if (c0 < 0) {
        c0 = 0;
        w = 0.f;
    }
    if (c0 >= C - 1) {
        c0 = C - 1;
        w = 0.f;
    }
}
// (1 - w) a + w b, rounded as: the first product, then one fused multiply-add
__device__ __forceinline__ float prolong_lerp(float a, float b, float w) {
    return __fmaf_rn(w, b, __fmul_rn(__fsub_rn(1.f, w), a));
}
// coarse column c of yc (Xc x Yc x Zc, x fastest) interpolated in y and z
__device__ __forceinline__ float prolong_col(const float* yc, int Xc, int Yc, int c, int y0, int y1, float wy, int z0,
                                             int z1, float wz) {
    const float a0 = prolong_lerp(yc[((size_t)z0 * Yc + y0) * Xc + c], yc[((size_t)z0 * Yc + y1) * Xc + c], wy);
    const float a1 = prolong_lerp(yc[((size_t)z1 * Yc + y0) * Xc + c], yc[((size_t)z1 * Yc + y1) * Xc + c], wy);
    return prolong_lerp(a0, a1, wz);
}
__device__ __forceinline__ float prolong_mix(float v0, float v1, float wx) { return prolong_lerp(v0, v1, wx); }

// per-cell flag bits: open faces of the cell, Poisson unknown, fluid
enum : uint8_t {
    F_E = 1, F_W = 2, F_N = 4, F_S = 8, F_T = 16, F_B = 32, F_UNK = 64, F_FLUID = 128
};

struct Dom {
    int nx, ny, nz;
    int px, py;                 // row pitch (elements), rows per plane (ny + 2)
    long long plane;            // px * py
    int perx, pery, perz;       // periodic axes
    __host__ __device__ __forceinline__ long long at(int i, int j, int k) const {
        return ((long long)k * py + j) * px + (i + OX);
    }
    __host__ __device__ __forceinline__ long long total() const { return plane * (nz + 2); }
};

// FP64 scalars produced and consumed on the device
struct Scalars {
    double rhs_mean;        // dz-weighted fluid mean of div(u*)/dt
    double rhs2;            // sum (rhs - mean)^2 over unknowns
    double res2;            // sum r^2 over unknowns
    double rel;             // sqrt(res2 / rhs2)
    double p_mean;          // dz-weighted fluid mean of p
    double q_in, q_out;     // volume fluxes after the outflow correction
    double mass_factor;     // Q_in / Q_out
    int converged;          // rel <= tol
    int nonfinite;          // a norm was NaN/Inf
    int sweeps;             // sweeps done in the current solve
    int batches;            // FP64 refinements done in the current solve
    long long step;         // time-step counter (read by bondv1 noise and adam)
    int noconv_any;         // sticky: a solve ended above tol since the last reset
    int zflag;              // 1: the correction is zero (a refinement just folded it in)
    int since;              // sweeps since the last refinement
    int refine;             // the last estimate asked for a refinement
    double est;             // FP32-arithmetic estimate of the relative residual
    double rho_ref;         // FP64 relative residual at the last refinement
    int done;               // the current solve has finished (kernels of a chunk exit early)
    int zcopy;              // zflag as it was before a network step wrote into the correction
    int timeout;            // a bounded device-side wait gave up (sticky until reported)
    int qpend;              // overlapped network correction: a prediction waits to be applied
};

// A refinement (FP64 accumulate + true residual) is taken when the cheap
// estimate reaches tol, has dropped kRefineDrop below the last true residual,
// kRefineEvery sweeps have passed, or the sweep budget is used up.
constexpr double kRefineDrop = 1e-3;
constexpr int kRefineEvery = 2000;

// what the residual kernel does with the solve's bookkeeping and, inside a
// CUDA graph, with the conditional nodes of the SOR loop
// What the residual kernels do with the solve's bookkeeping.
//   RES_INIT   first residual of a solve: resets the counters and `done`
//   RES_LOOP   refinement after an estimate asked for it
//   RES_FIXED  the single residual after a fixed number of sweeps
enum ResMode { RES_INIT = 0, RES_LOOP = 1, RES_FIXED = 2 };
struct CondArgs {
    int mode;               // ResMode
    int n;                  // sweeps in the batch just finished (estimate / fixed)
    int limit;              // sweep budget of the solve (max_sweeps)
    int gate;               // 1: run only while !done and a refinement was asked for; 2: only while !done
    int force;              // estimate: ask for a refinement whatever the estimate says
    double tol;
    int* done_host;         // mapped host copy of `done` (nullable)
};

// constant per-run data in the compute type
template <typename T>
struct Geo {
    Dom d;
    T dx, dy, rdx, rdy, dt, nu, omega;
    T cx, cy;               // 1/dx^2, 1/dy^2
    const T* dz;            // [nz+2] padded cell heights
    const T* dzs;           // [nz+2] centre-to-centre spacing dzs_k = (dz_k + dz_{k+1})/2
    const T* cT;            // [nz+2] 1/(dz_k dzs_k)
    const T* cB;            // [nz+2] 1/(dz_k dzs_{k-1})
    const T* delta2;        // [nz+2] (Cs Delta_k)^2
    const T* rdz;           // [nz+2] 1 / dz_k
    const T* rdzs;          // [nz+2] 1 / dzs_k
    const double* dz64;     // [nz+2]
    double dx64, dy64, cx64, cy64;
    const double* dzs64;    // [nz+2]
    const double* cT64;     // [nz+2]
    const double* cB64;     // [nz+2]
    const uint8_t* flags;   // padded cell flags
    const T* cn1;           // [nz+2][64] cn1 over (plane, open-face mask); FP32 grids only (else null)
    const T* ctab;          // [nz+2+16][68] per-plane rows of the column-walk sweeps: cn1[64], cT, cB, 0, 0
                            // (wrapped on a periodic z axis, else clamped); FP32 grids only (else null)
    const double* diag64;   // [nz+2][64] FP64 diagonal of the Poisson operator over (plane, open-face mask)
};

struct Reduce {
    double* partials;       // [3 * max_blocks]
    unsigned* counter;      // zero between launches
    Scalars* sc;
};

// inflow profile series in time (n = 0: the fixed profile is used)
struct InflowSeries {
    const double* p;        // [n][nz+2] profiles (level k at index k)
    const double* t;        // [n] increasing times (s)
    int n;
    double dt;
};

// launchers (les_kernels.cu); each returns the number of kernels launched
template <typename T> int launch_bc(const Geo<T>& g, T* u, T* v, T* w, const double* inflow,
                                    const InflowSeries& ser, double turb, uint64_t seed, const Scalars* sc,
                                    cudaStream_t s);
template <typename T> int launch_nut(const Geo<T>& g, const T* u, const T* v, const T* w, T* nut,
                                     cudaStream_t s);
template <typename T> int launch_momentum(const Geo<T>& g, const T* u, const T* v, const T* w,
                                          const T* nut, T* fu, T* fv, T* fw, T* us, T* vs, T* ws,
                                          const Scalars* sc, cudaStream_t s);
template <typename T> int launch_outflow(const Geo<T>& g, const T* u, T* us, T* vs, T* ws, const Reduce& red,
                                         cudaStream_t s);
template <typename T> int launch_rhs(const Geo<T>& g, const T* us, const T* vs, const T* ws, T* rhs,
                                     double vfluid, const Reduce& r, cudaStream_t s);
template <typename T> int launch_rhs_mean(const Geo<T>& g, T* rhs, double vfluid, const Reduce& r,
                                          cudaStream_t s);
// zero_start: 0 continue from d, 1 treat d as zero, 2 read the device flag sc->zflag
template <typename T> int launch_sor_sweep(const Geo<T>& g, T* dl, const T* r, int zero_start, const Scalars* sc,
                                           cudaStream_t s);
template <typename T> int launch_accum(const Geo<T>& g, double* ph, const T* dl, const Scalars* sc, int gate,
                                       cudaStream_t s);
template <typename T> int launch_residual64(const Geo<T>& g, const double* ph, const T* rhs, T* r,
                                            double vfluid, const Reduce& red, CondArgs ca, cudaStream_t s);
template <typename T> int launch_sor_est(const Geo<T>& g, const T* dl, const T* r, T* rout, const Reduce& red, CondArgs ca,
                                         cudaStream_t s);
int reduce_blocks(const Dom& d);
template <typename T> int launch_project(const Geo<T>& g, const T* us, const T* vs, const T* ws,
                                         T* u, T* v, T* w, const double* ph_in, double* ph_out,
                                         Scalars* sc, cudaStream_t s);
template <typename T> int launch_rhs_eff(const Geo<T>& g, const T* rhs, T* out, const Scalars* sc,
                                         cudaStream_t s);

template <typename T> int launch_gauge(const Geo<T>& g, const double* p_in, double* p_out,
                                       const Scalars* sc, cudaStream_t s);

// fused SOR sweep (les_sor.cu): tile shape index into kSorTiles and k-chunk
// ---------------------------------------------------------------------------
// ensembles: the per-member arguments of the batched kernels, passed as one
// __grid_constant__ kernel parameter (< 32 KB)
constexpr int kMaxMembers = 64;
template <typename T>
struct EnsMember {
    Geo<T> g;
    T* dl[2];               // SOR correction (ping-pong)
    T* rr;                  // residual of the FP64 pressure (field type)
    const T* rhs;
    double* ph;             // FP64 pressure of the current step
    double vfluid;
    double tol;
    int limit;              // sweep budget of the member's solve
    Reduce red;             // the member's partials, counter and scalars
    int sgrid[3];           // sweep tiles of the ensemble tile shape
    int egrid[3];           // estimate blocks
    int agrid[3];           // accumulate blocks (32 x 8 threads, one plane per block)
    int rblocks;            // residual blocks (grid-stride)
    T* rcur;                // residual copy for the network correction (null without one)
};
template <typename T>
struct EnsTab {
    int n;
    int tile;                       // ensemble row tile 0..kNumEnsTiles-1
    int sbeg[kMaxMembers + 1];      // first flattened item of each member, per kernel kind
    int ebeg[kMaxMembers + 1];
    int abeg[kMaxMembers + 1];
    int rbeg[kMaxMembers + 1];
    int tbeg[kMaxMembers + 1];      // first item of each member in the batched TMA sweep's list
    int* ndone;                     // members whose solve has ended (device counter)
    int* all_done_host;             // mapped host flag set when ndone reaches n
    EnsMember<T> m[kMaxMembers];
};
static_assert(sizeof(EnsTab<float>) < 32000, "ensemble table must fit in the kernel parameter space");
constexpr int kFirstRowTile = 12, kNumEnsTiles = 5;
constexpr int kEstChunk = 8;       // planes per thread in the estimate and line-search kernels

struct SorTile { int tx, ty, tz; };   // tz = 0: k-marching column tile
struct SorCfg { int tile; int kc; };   // tile < 0: two in-place half-sweep kernels
extern const SorTile kSorTiles[];
extern const int kNumSorTiles;
// ensemble launchers: the batched sweep (les_sor.cu) and the batched estimate /
// refinement (les_kernels.cu); one launch each covers every member
SorTile ens_tile_shape(int t);
int ens_rows_smem(int t);
int launch_sor_ens(const EnsTab<float>& tab, int in, int zero, int ctas, cudaStream_t s);
int launch_est_ens(const EnsTab<float>& tab, int dcur, const CondArgs& ca, cudaStream_t s);
int launch_refine_ens(const EnsTab<float>& tab, int dcur, const CondArgs& ca, cudaStream_t s);
template <typename T> int launch_sor_fused(const Geo<T>& g, const T* din, T* dout, const T* r, int zero_start,
                                           const Scalars* sc, SorCfg cfg, cudaStream_t s);

template <typename T> cudaError_t sor_prepare();

// TMA variants (les_sor_tma.cu), FP32; tile indices kFirstTmaTile ..
// kFirstTmaTile + kNumTmaTiles - 1: the first kNumTmaBlockTiles are one CTA
// per block (any boundary conditions), the next four persistent
// double-buffered (no periodic axis), the next four k-marching columns with
// a plane pipeline (any boundary conditions; kc = planes per chunk), the
// last six one CTA per block with the column-walk update (any boundary
// conditions)
constexpr int kFirstTmaTile = 17;
constexpr int kNumTmaTiles = 18;
constexpr int kNumTmaBlockTiles = 4;
constexpr int kFirstMarchCfg = 8;
constexpr int kFirstColCfg = 12;
extern const int kTmaCfg[kNumTmaTiles][3];
struct TmaMaps {
    CUtensorMap d[2], r, f;
    const float* dptr[2];       // the arrays behind the maps (periodic halo images)
    const float* rptr;
};
bool tma_supported(const Dom& d);
bool pipe_supported(const Dom& d);
cudaError_t tma_prepare();
bool tma_encode(const Dom& d, float* dl0, float* dl1, float* rr, uint8_t* flags, TmaMaps* maps);
// pre = 1: the kernel before this one in the stream is a sweep of the same
// batch (the column-walk tiles then copy r, flags and coefficients before
// the dependency wait)
int launch_sor_tma(const Geo<float>& g, const TmaMaps* maps, const float* cn1tab, int cfg, int kc, int in,
                   float* dout, int zero, Scalars* sc, cudaStream_t s, int pre = 0);
int launch_cn1_table(const Geo<float>& g, float* tab, cudaStream_t s);
// the column-walk sweeps' coefficient rows from the cn1 table ((nz + 2 + 16) rows of 68 floats)
int launch_col_table(const Geo<float>& g, const float* cn1tab, float* tab, cudaStream_t s);
constexpr int kColTableRows = 16;    // rows past plane nz + 1
// batched TMA sweep of an ensemble (les_sor_tma.cu): the 28 x 8 x 8 blocks of
// every member in one persistent launch; maps = 4 tensor maps per member
// (d[0], d[1], r, flags) in global memory, encoded by tma_encode_member
constexpr int kEnsTmaBy = 8, kEnsTmaBz = 8;
bool tma_encode_member(const Dom& d, float* dl0, float* dl1, float* rr, const uint8_t* flags, CUtensorMap* out4);
int launch_sor_tma_ens(const EnsTab<float>& tab, const CUtensorMap* maps, int in, int zero, int ctas,
                       cudaStream_t s);
int sor_tma_ens_resident();     // resident CTAs of the batched TMA sweep on this device
// the estimate of an FP32 grid with no periodic axis from TMA tiles (the
// cells, arithmetic and sums of launch_sor_est, so the same result): maps
// from tma_encode_est (d[0], d[1], r, flags); dcur selects d
bool tma_encode_est(const Dom& d, float* dl0, float* dl1, float* rr, const uint8_t* flags, CUtensorMap* out4);
// The network's pooled input, formed by that estimate when it is given one
// (the network correction that follows the estimate then skips its pooling
// kernel): the residual r_out and the unknown mask averaged over stride-s
// cubes (s = 4 or 8, which tile the estimate's 32 x 8 x 8 blocks), into rc
// and mask (coarse volume xc * yc * zc, x fastest), and scal[0] = the
// mask-weighted RMS of rc, scal[1] = the sum of the mask, both FP64.
struct EstPool {
    float* rc = nullptr;       // null: the estimate does not pool
    float* mask = nullptr;
    double* scal = nullptr;
    int s = 0, xc = 0, yc = 0, zc = 0;
};
int launch_sor_est_tma(const Geo<float>& g, const CUtensorMap* maps4, int dcur, float* rout, const Reduce& red,
                       CondArgs ca, cudaStream_t s, const EstPool& pool = EstPool{});
// the plain-SOR solve of an ensemble as one persistent cooperative launch
// (les_kernels.cu); bar: 2 zeroed unsigned of grid-barrier state, err: a
// zeroed device flag set when a bounded wait gave up; returns the launches
// (1), or -1 when the device cannot run it
int launch_ens_persist(const EnsTab<float>& tab, const CUtensorMap* maps, int cycle, int batches, const CondArgs& ca,
                       unsigned* bar, int* err, cudaStream_t s);
int ens_persist_grid();
template <typename T> int launch_diag_table(const Geo<T>& g, double* tab, cudaStream_t s);
// comparison of SOR variants (les_sor_compare)
template <typename T> int launch_cmp_residual(const Geo<T>& g, const double* p, const double* b, T* r,
                                              const Reduce& red, double* out, cudaStream_t s);
template <typename T> int launch_cmp_add(const Geo<T>& g, const double* p0, const T* dv, int stride, double* pn,
                                         size_t n, cudaStream_t s);
template <typename T> int launch_twin_half(const Geo<T>& g, void* tw, const T* r, int nrd, T omega, cudaStream_t s);
int launch_wait_selftest(unsigned long long limit_ns, int* status, cudaStream_t s);

// learned warm start (les_kernels.cu): energy-norm line search along q and p += alpha q
// (dl null: p_h += alpha q at the start of a solve; dl set: inside the loop the
// SOR correction takes the step)
template <typename T> int launch_warm(const Geo<T>& g, const T* r, const float* q, double* ph, T* dl, double* alpha,
                                      const Reduce& red, cudaStream_t s);
// the same with the network's prolongation folded into the line search: yc
// is the coarse output (cell-centred, stride st in {1, 2, 4, 8}); the line
// search prolongs it on the fly (the arithmetic of the stand-alone
// prolongation kernel) and leaves the dense fine correction in q for the step
template <typename T> int launch_warm_coarse(const Geo<T>& g, const T* r, const float* yc, int st, float* q,
                                             double* ph, T* dl, double* alpha, const Reduce& red, cudaStream_t s);
// the overlapped correction inside the loop: the line search of the pending
// prediction q against the current residual r, then d += alpha q and
// r -= alpha A q (r becomes the residual after the step: the next
// prediction's input); both kernels return at once unless sc->qpend is set
template <typename T> int launch_warm_pending(const Geo<T>& g, T* r, const float* q, T* dl, double* alpha,
                                              const Reduce& red, cudaStream_t s);
int launch_set_flag(int* flag, int value, const int* gate, cudaStream_t s);
// training-pair recording: what 0 = ph - ph0 into out, 1 = unknown mask into out
template <typename T> int launch_record(const Geo<T>& g, const double* ph, const double* ph0, T* out, int what,
                                        cudaStream_t s);
int launch_count_unknowns(const Dom& d, const uint8_t* flags, unsigned long long* out, cudaStream_t s);

int max_reduce_blocks(const Dom& d);

}  // namespace les

struct les_s;
namespace les {
// ensemble support (les_api.cu): the members are ordinary domain handles
int member_check(les_s* h, char* why, size_t n);          // 0 if h can join an ensemble
void member_fill(les_s* h, EnsMember<float>& M, int ens_tile, int parity);
int member_parity(const les_s* h);                        // which pressure buffer is current
int member_begin(les_s* h, cudaStream_t s);               // clears the sticky non-convergence flag
int member_check_every(const les_s* h);
int member_max_sweeps(const les_s* h);
cudaStream_t member_stream(const les_s* h);
int member_prefix(les_s* h, cudaStream_t s);              // bondv1 .. rhs of the step; launches, or < 0 on error
int member_finish(les_s* h, cudaStream_t s);              // velnw, buffer flip, step counter
int member_stats(les_s* h, les_stats_t* st);              // reads the scalars back; returns the status
void member_set_dcur(les_s* h, int dcur);
int member_sweep(les_s* h, int in, int zero, cudaStream_t s);   // one sweep d[in] -> d[1-in], own kernel
int member_autotune(les_s* h, int sweeps);                       // the member's own sweep configuration
int* member_done_flag(les_s* h);                           // device address of the member's `done`
// the learned correction of a member (set with les_set_warmstart / les_set_net_schedule)
bool member_net_on(const les_s* h);                        // network inside the solve loop
int member_net_every(const les_s* h);
int member_net_prepare(les_s* h);                          // workspace, before a capture
long long member_net_generation(const les_s* h);
int member_net_start(les_s* h, cudaStream_t s);           // step at the start of the solve
int member_net_loop(les_s* h, cudaStream_t s);            // step inside the loop (done-gated)
}  // namespace les

struct les_net_s;
namespace les {
// network prediction on a solver grid (les_net.cu): the padded residual and
// the unknown flags in, the correction direction as a dense (nz, ny, nx)
// array out (zero off the unknowns)
// (`gate` nullable: every kernel returns at once while *gate != 0)
// (after_pool, nullable: recorded on s once the residual has been read)
// (fold: on the tcgen05 engine the packing runs inside the first
// convolution and the head inside the last; false keeps their own kernels,
// which compute the same values)
int net_predict(les_net_s* n, const Dom& d, const float* r_padded, const uint8_t* flags, float* out_dense,
                cudaStream_t s, const int* gate = nullptr, cudaEvent_t after_pool = nullptr, bool fold = true,
                bool pooled = false);
// the same without the prolongation: the coarse output is left in
// net_coarse_out(n) (stride net_stride(n)) for a line search that prolongs it
// on the fly (launch_warm_coarse)
int net_predict_coarse(les_net_s* n, const Dom& d, const float* r_padded, const uint8_t* flags, cudaStream_t s,
                       const int* gate = nullptr, bool pooled = false);
// where the estimate before a correction may leave the network's pooled input
// (EstPool above) for solver grid d: false when the network pools on its own
// (a stride other than 4 or 8, or a coarse grid beyond the pooling kernel's
// size); sizes the workspace first.  `pooled` in net_predict /
// net_predict_coarse then skips the pooling kernel.
bool net_pool_target(les_net_s* n, const Dom& d, EstPool* out);
const float* net_coarse_out(const les_net_s* n);
int net_stride(const les_net_s* n);
int net_launches(const les_net_s* n);
// size the network's workspace for a solver grid ahead of a graph capture; the
// generation changes whenever the workspace is reallocated (captured graphs
// holding the old buffers must then be rebuilt)
int net_prepare(les_net_s* n, const Dom& d, long long* generation);
long long net_generation(const les_net_s* n);
// the prediction with the coarse network as one cooperative persistent launch
// (pool and prolongation as full-grid kernels around it); LES_EINVAL if the
// device cannot run it
int net_predict_persistent(les_net_s* n, const Dom& d, const float* r_padded, const uint8_t* flags, float* q_dense,
                           Scalars* sc, const int* gate, cudaStream_t s);
int net_persistent_launches();
}  // namespace les
