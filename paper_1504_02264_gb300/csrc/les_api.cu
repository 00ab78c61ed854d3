// Host side of the C ABI declared in include/les.h: handle, validation,
// device allocation, host <-> device staging and the per-step launch order.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <vector>

#include <cuda_profiler_api.h>

#include "../../include/les.h"
#include "les_internal.cuh"

using namespace les;

namespace {

const char* kVersion = "les-gb300 0.1 (sm_103a)";

// packing kernels between the padded device layout and the dense I/O layout
template <typename S, typename T>
__global__ void k_pack(Dom d, const S* src, T* dst, int i0, int j0, int k0, int ni, int nj, int nk) {
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long n = (long long)ni * nj * nk;
    if (q >= n) return;
    int i = (int)(q % ni);
    long long r = q / ni;
    int j = (int)(r % nj);
    int k = (int)(r / nj);
    dst[q] = (T)src[d.at(i0 + i, j0 + j, k0 + k)];
}
template <typename S, typename T>
__global__ void k_unpack(Dom d, const S* src, T* dst, int i0, int j0, int k0, int ni, int nj, int nk) {
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long n = (long long)ni * nj * nk;
    if (q >= n) return;
    int i = (int)(q % ni);
    long long r = q / ni;
    int j = (int)(r % nj);
    int k = (int)(r / nj);
    dst[d.at(i0 + i, j0 + j, k0 + k)] = (T)src[q];
}

// open-face flags from the padded solid mask (ghost cells are fluid and are
// never consulted across a non-periodic domain face)
__global__ void k_flags(Dom d, const uint8_t* solid, uint8_t* flags) {
    int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    int k = blockIdx.z + 1;
    if (i > d.nx || j > d.ny) return;
    auto fl = [&](int a, int b, int c) -> bool {
        if (d.perx) a = a < 1 ? a + d.nx : (a > d.nx ? a - d.nx : a);
        if (d.pery) b = b < 1 ? b + d.ny : (b > d.ny ? b - d.ny : b);
        if (d.perz) c = c < 1 ? c + d.nz : (c > d.nz ? c - d.nz : c);
        if (a < 1 || a > d.nx || b < 1 || b > d.ny || c < 1 || c > d.nz) return false;
        return solid[d.at(a, b, c)] == 0;
    };
    uint8_t f = 0;
    if (fl(i, j, k)) {
        f |= F_FLUID;
        if (fl(i + 1, j, k)) f |= F_E;
        if (fl(i - 1, j, k)) f |= F_W;
        if (fl(i, j + 1, k)) f |= F_N;
        if (fl(i, j - 1, k)) f |= F_S;
        if (fl(i, j, k + 1)) f |= F_T;
        if (fl(i, j, k - 1)) f |= F_B;
        if (f & (F_E | F_W | F_N | F_S | F_T | F_B)) f |= F_UNK;
    }
    flags[d.at(i, j, k)] = f;
}

}  // namespace

struct les_s {
    les_grid_t g;
    std::vector<double> dz;        // [nz]
    std::vector<double> inflow;    // [nz+2] padded
    Dom d;
    int prec;
    size_t es;                     // element size
    size_t n;                      // elements per padded array
    // device arrays (element type per precision)
    void *u = nullptr, *v = nullptr, *w = nullptr, *us = nullptr, *vs = nullptr, *ws = nullptr;
    void *fu = nullptr, *fv = nullptr, *fw = nullptr, *nut = nullptr, *rhs = nullptr, *tmp = nullptr;
    double* ph[2] = {nullptr, nullptr};   // FP64 pressure (velnw writes the gauged copy to the other)
    void* dl[2] = {nullptr, nullptr};     // SOR correction (ping-pong for the fused sweep)
    void* rr = nullptr;                   // its FP64-formed right-hand side
    SorCfg sor = {6, 0};                  // fused kernel, 32 x 8 x 4 blocks (les_autotune_sor refines)
    void* stage = nullptr;         // dense I/O staging
    size_t stage_elems = 0;
    uint8_t* flags = nullptr;
    void *kdz = nullptr, *kdzs = nullptr, *kcT = nullptr, *kcB = nullptr, *kdel = nullptr;
    void *krdz = nullptr, *krdzs = nullptr;   // reciprocals of dz and dzs
    double* dz64 = nullptr;
    double *dzs64 = nullptr, *cT64 = nullptr, *cB64 = nullptr;
    double* inflow64 = nullptr;
    double* partials = nullptr;
    unsigned* counter = nullptr;
    Scalars* sc = nullptr;
    Scalars* sc_host = nullptr;    // pinned
    cudaStream_t stream = nullptr;
    int cur = 0;
    long long step = 0;
    double vfluid = 0.0;
    long long launches = 0;
    std::vector<void*> allocs;
    // CUDA graph of one step per pressure-buffer parity
    bool use_graph = true;
    bool graph_ok[2] = {false, false};
    long long graph_launches[2] = {0, 0};  // kernels in each fixed-sweep step graph
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    cudaStream_t cap[1] = {nullptr};
    cudaEvent_t chunk_ev[2] = {nullptr, nullptr};
    int* done_host = nullptr;             // mapped pinned copy of the device `done` flag
    int* done_dev = nullptr;              // its device address
    int dcur = 0;                         // buffer holding the current SOR correction
    bool graph_failed = false;            // graph build failed once; host-driven loop in use
    bool last_graph = false;              // the last les_step ran as graphs
    TmaMaps tma[kNumTmaTiles];            // tensor maps of the TMA sweep (FP32, no periodic axis)
    bool tma_ok = false;
    bool pipe_ok = false;                 // persistent TMA tiles (no periodic axis)
    CUtensorMap est_maps[4];              // the TMA estimate's tiles (FP32, no periodic axis)
    bool est_tma = false;
    float* cn1tab = nullptr;              // cn1 over (plane, open-face mask) for the pipelined sweep
    float* coltab = nullptr;              // per-plane coefficient rows of the column-walk sweeps
    double* diag64 = nullptr;             // FP64 diagonal over (plane, open-face mask), the residual's
    // les_sor_compare scratch (allocated on first use): p0, rhs, p0 + d (FP64,
    // padded), the four norms, and the twinned pair array of the correction
    double* cmp_p0 = nullptr;
    double* cmp_b = nullptr;
    double* cmp_pn = nullptr;
    double* cmp_out = nullptr;
    void* twin = nullptr;
    // learned warm start and training-pair recording
    int warm = LES_WARM_PREV;
    les_net_s* net = nullptr;
    float* pred = nullptr;                // dense (nz, ny, nx) predicted correction
    void* rcur = nullptr;                 // current residual written by the estimate (network input in the loop)
    double* warm_scal = nullptr;          // [0] input scale, [1] line-search step
    double n_unk = 0.0;                   // number of Poisson unknowns
    int net_every = 0;                    // sweeps between network corrections inside a solve (0: start only)
    // inflow profile series in time (device; nseries = 0: the fixed profile)
    double* series_p = nullptr;
    double* series_t = nullptr;
    int nseries = 0, series_cap = 0;
    long long net_gen = -1;               // network workspace generation the chunk graphs were captured with
    int net_kernels = LES_NET_KERNELS_FOLDED;   // how a correction's kernels are laid out (les_set_net_kernels)
    bool net_own_pool = false;                  // the network pools on its own (LES_NET_KERNELS_OWN_POOL)
    long long net_chunk_launches = 0;           // network kernels of one correction in the chunk graphs
    bool net_persistent = false;          // coarse network as one cooperative launch
    bool net_async = false;               // graph loop: each prediction overlaps the next batch of sweeps
    cudaStream_t s2 = nullptr;            // its stream, and the events that order it with the loop
    cudaEvent_t ev_fork = nullptr, ev_pool = nullptr, ev_q = nullptr;
    bool net_start = true;                // also correct at the start of each solve
    bool record = false;
    int rec_after = 0;                    // record at the first refinement after this many sweeps
    bool rec_taken = false;               // the current solve has taken its pair's input
    bool rec_valid = false;               // the last solve recorded a complete pair
    double* rec_p0 = nullptr;             // pressure before the last solve
    void* rec_r0 = nullptr;               // initial residual of the last solve
    void* rec_delta = nullptr;            // correction applied by the last solve
    void* rec_netin = nullptr;            // residual the start-of-solve network correction saw
    float* rec_netq = nullptr;            // its prediction q (dense (nz, ny, nx))
    bool net_taken = false;               // a start-of-solve prediction has been recorded
    // phase timing
    bool timing = false;
    cudaEvent_t ev[8] = {};
    les_timing_t tm = {};
    char err[512] = {0};
};

namespace {

char g_static_err[512] = "";

int fail(les_s* h, int code, const char* fmt, ...) {
    char* buf = h ? h->err : g_static_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return code;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(h, LES_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

int dalloc(les_s* h, void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return fail(h, LES_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    h->allocs.push_back(*p);
    e = cudaMemsetAsync(*p, 0, bytes, h->stream);
    if (e != cudaSuccess) return fail(h, LES_ECUDA, "cudaMemset failed: %s", cudaGetErrorString(e));
    return LES_OK;
}

// staggering: 0 cell, 1 x-face, 2 y-face, 3 z-face
void io_box(const les_s* h, int stag, int& i0, int& j0, int& k0, int& ni, int& nj, int& nk) {
    ni = h->g.nx + (stag == 1);
    nj = h->g.ny + (stag == 2);
    nk = h->g.nz + (stag == 3);
    i0 = stag == 1 ? 0 : 1;
    j0 = stag == 2 ? 0 : 1;
    k0 = stag == 3 ? 0 : 1;
}

size_t io_elems(const les_s* h, int stag) {
    int i0, j0, k0, ni, nj, nk;
    io_box(h, stag, i0, j0, k0, ni, nj, nk);
    return (size_t)ni * nj * nk;
}

// host (type T, dense) -> device array of type D (padded)
template <typename T, typename D = T>
int upload(les_s* h, void* dev, int stag, const void* host, size_t stage_off) {
    int i0, j0, k0, ni, nj, nk;
    io_box(h, stag, i0, j0, k0, ni, nj, nk);
    size_t n = (size_t)ni * nj * nk;
    T* st = (T*)h->stage + stage_off;
    CK(cudaMemcpyAsync(st, host, n * sizeof(T), cudaMemcpyHostToDevice, h->stream));
    k_unpack<T, D><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(h->d, st, (D*)dev, i0, j0, k0, ni, nj, nk);
    h->launches++;
    CK(cudaGetLastError());
    return LES_OK;
}

// device array of type D (padded) -> host (type T, dense)
template <typename T, typename D = T>
int download(les_s* h, const void* dev, int stag, void* host, size_t stage_off) {
    int i0, j0, k0, ni, nj, nk;
    io_box(h, stag, i0, j0, k0, ni, nj, nk);
    size_t n = (size_t)ni * nj * nk;
    T* st = (T*)h->stage + stage_off;
    k_pack<D, T><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(h->d, (const D*)dev, st, i0, j0, k0, ni, nj, nk);
    h->launches++;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(host, st, n * sizeof(T), cudaMemcpyDeviceToHost, h->stream));
    return LES_OK;
}

template <typename T>
Geo<T> geo(les_s* h) {
    Geo<T> g;
    g.d = h->d;
    g.dx = (T)h->g.dx;
    g.dy = (T)h->g.dy;
    g.rdx = (T)(1.0 / h->g.dx);
    g.rdy = (T)(1.0 / h->g.dy);
    g.dt = (T)h->g.dt;
    g.nu = (T)h->g.nu;
    g.omega = (T)h->g.omega;
    g.cx = (T)(1.0 / (h->g.dx * h->g.dx));
    g.cy = (T)(1.0 / (h->g.dy * h->g.dy));
    g.dz = (const T*)h->kdz;
    g.dzs = (const T*)h->kdzs;
    g.cT = (const T*)h->kcT;
    g.cB = (const T*)h->kcB;
    g.delta2 = (const T*)h->kdel;
    g.rdz = (const T*)h->krdz;
    g.rdzs = (const T*)h->krdzs;
    g.dz64 = h->dz64;
    g.dx64 = h->g.dx;
    g.dy64 = h->g.dy;
    g.cx64 = 1.0 / (h->g.dx * h->g.dx);
    g.cy64 = 1.0 / (h->g.dy * h->g.dy);
    g.dzs64 = h->dzs64;
    g.cT64 = h->cT64;
    g.cB64 = h->cB64;
    g.flags = h->flags;
    g.cn1 = std::is_same<T, float>::value ? (const T*)h->cn1tab : nullptr;
    g.ctab = std::is_same<T, float>::value ? (const T*)h->coltab : nullptr;
    g.diag64 = h->diag64;
    return g;
}

Reduce reducer(les_s* h) { return Reduce{h->partials, h->counter, h->sc}; }

template <typename T>
int upload_table(les_s* h, void* dev, const std::vector<double>& v) {
    std::vector<T> t(v.begin(), v.end());
    CK(cudaMemcpyAsync(dev, t.data(), t.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LES_OK;
}

int fetch_scalars(les_s* h) {
    CK(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LES_OK;
}

void rec(les_s* h, int e) {
    if (h->timing) cudaEventRecord(h->ev[e], h->stream);
}
double elapsed(les_s* h, int a, int b) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev[a], h->ev[b]);
    return ms;
}

// press: SOR iterations under the stop rule.  The FP64 pressure ph[cur] is
// refined by batches of sweeps on the correction d (k_accum adds d, then
// k_residual64 forms the next right-hand side and the FP64 residual); the
// relative residual is tested after each batch of check_every sweeps and at
// max_sweeps, exactly where the sequential algorithm tests it.

// the estimate after a batch of sweeps: from TMA tiles on FP32 grids with no
// periodic axis, else the plain kernel (both give the same result)
// (pool, nullable: the TMA estimate also forms the network's pooled input there)
template <typename T>
int launch_estimate(les_s* h, const Geo<T>& g, T* rout, CondArgs ca, cudaStream_t st, const EstPool* pool = nullptr) {
    if constexpr (std::is_same<T, float>::value) {
        if (h->est_tma)
            return launch_sor_est_tma(g, h->est_maps, h->dcur, rout, reducer(h), ca, st, pool ? *pool : EstPool{});
    }
    return launch_sor_est<T>(g, (const T*)h->dl[h->dcur], (const T*)h->rr, rout, reducer(h), ca, st);
}

// n sweeps on the correction.  zero: 0 continue from d, 1 start from d = 0,
// 2 read the device flag.  The fused kernel ping-pongs between the two d
// buffers starting from dl[h->dcur]; the result's buffer index is returned
// (and becomes dcur).
template <typename T>
int run_sweeps(les_s* h, const Geo<T>& g, int n, int zero, long long& launched, cudaStream_t st) {
    T* rr = (T*)h->rr;
    if (h->sor.tile < 0) {
        for (int s = 0; s < n; ++s) launched += launch_sor_sweep<T>(g, (T*)h->dl[0], rr, s == 0 ? zero : 0, h->sc, st);
        return h->dcur = 0;
    }
    for (int s = 0; s < n; ++s) {
        const int in = h->dcur, out = 1 - h->dcur;
        if constexpr (std::is_same<T, float>::value) {
            if (h->sor.tile >= kFirstTmaTile) {
                launched += launch_sor_tma(g, h->tma, h->cn1tab, h->sor.tile - kFirstTmaTile, h->sor.kc, in,
                                           (float*)h->dl[out], s == 0 ? zero : 0, h->sc, st, s > 0 ? 1 : 0);
                h->dcur = out;
                continue;
            }
        }
        launched += launch_sor_fused<T>(g, (const T*)h->dl[in], (T*)h->dl[out], rr, s == 0 ? zero : 0, h->sc, h->sor,
                                        st);
        h->dcur = out;
    }
    return h->dcur;
}

CondArgs cond_args(const les_s* h, int mode, int n, int gate) {
    CondArgs ca{};
    ca.mode = mode;
    ca.n = n;
    ca.limit = h->g.max_sweeps;
    ca.gate = gate;
    ca.tol = h->g.tol;
    ca.done_host = h->done_dev;
    return ca;
}

// Move p along the network's predicted correction q = Net(r / rms(r)) with
// the energy-norm line search, then form the FP64 residual again (`mode` is
// RES_INIT at the start of a solve, RES_LOOP inside it, where the new
// residual may already pass the stop test).
// the network's prediction q of the correction for residual r: the coarse
// network as one cooperative launch when the device can, else per layer
int predict(les_s* h, const float* r, cudaStream_t st, const int* gate, bool pooled = false) {
    if (h->net_persistent) {
        int rc = net_predict_persistent(h->net, h->d, r, h->flags, h->pred, h->sc, gate, st);
        if (rc == LES_OK) {
            h->launches += net_persistent_launches();
            return LES_OK;
        }
        if (rc != LES_EINVAL) return fail(h, rc, "persistent network prediction failed");
    }
    int rc = net_predict(h->net, h->d, r, h->flags, h->pred, st, gate, nullptr,
                         h->net_kernels != LES_NET_KERNELS_LAYERS, pooled);
    if (rc) return fail(h, rc, "network prediction failed");
    h->launches += net_launches(h->net);
    return LES_OK;
}

// The prediction for residual r and the energy-norm step along it: into the
// FP64 pressure ph (dl null) or into the SOR correction dl.  Folded kernels
// (default): the prolongation runs inside the line search, which leaves the
// fine correction in h->pred for the step; otherwise (the persistent network,
// or the stand-alone kernels) the prolongation has its own kernel first.
// (pooled: the estimate before this call left the network's pooled input)
template <typename T>
int net_step(les_s* h, const Geo<T>& g, const T* r, double* ph, T* dl, cudaStream_t st, const int* gate,
             bool pooled = false) {
    if (h->net_kernels == LES_NET_KERNELS_FOLDED) {
        int rc = net_predict_coarse(h->net, h->d, (const float*)r, h->flags, st, gate, pooled);
        if (rc) return fail(h, rc, "network prediction failed");
        h->launches += net_launches(h->net);
        h->launches += launch_warm_coarse<T>(g, r, net_coarse_out(h->net), net_stride(h->net), h->pred, ph, dl,
                                             h->warm_scal + 1, reducer(h), st);
        return LES_OK;
    }
    int rc = predict(h, (const float*)r, st, gate, pooled);
    if (rc) return rc;
    h->launches += launch_warm<T>(g, r, h->pred, ph, dl, h->warm_scal + 1, reducer(h), st);
    return LES_OK;
}

template <typename T>
int net_correct(les_s* h, const Geo<T>& g, cudaStream_t st) {
    if (h->record) CK(cudaMemcpyAsync(h->rec_netin, h->rr, h->n * h->es, cudaMemcpyDeviceToDevice, st));
    int rc = net_step<T>(h, g, (const T*)h->rr, h->ph[h->cur], (T*)nullptr, st, nullptr);
    if (rc) return rc;
    if (h->record) {
        CK(cudaMemcpyAsync(h->rec_netq, h->pred, (size_t)h->g.nx * h->g.ny * h->g.nz * sizeof(float),
                           cudaMemcpyDeviceToDevice, st));
        h->net_taken = true;
    }
    h->launches += launch_residual64<T>(g, h->ph[h->cur], (const T*)h->rhs, (T*)h->rr, h->vfluid, reducer(h),
                                        cond_args(h, RES_INIT, 0, 0), st);
    CK(cudaGetLastError());
    return LES_OK;
}

// The network correction inside the solve loop: q = Net(r) from the residual
// the last estimate stored, the energy-norm step into the FP32 SOR correction
// (no FP64 pass: the next refinement folds it into p).  `gated`: captured in a
// chunk graph, every kernel returns at once when the solve is done.
template <typename T>
int net_correct_loop(les_s* h, const Geo<T>& g, cudaStream_t st, bool gated, bool pooled = false) {
    int rc = net_step<T>(h, g, (const T*)h->rcur, nullptr, (T*)h->dl[h->dcur], st, gated ? &h->sc->done : nullptr,
                         pooled);
    if (rc) return rc;
    CK(cudaGetLastError());
    return LES_OK;
}

void record_start(les_s* h, cudaStream_t st) {
    cudaMemcpyAsync(h->rec_p0, h->ph[h->cur], h->n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(h->rec_r0, h->rr, h->n * h->es, cudaMemcpyDeviceToDevice, st);
    h->rec_taken = true;
}

// After the first FP64 residual of a solve: the cold start (p = 0) or the
// learned warm start, then the recording of the training pair's input when
// it is taken at the start.
template <typename T>
int solve_start(les_s* h, const Geo<T>& g, cudaStream_t st) {
    if (h->warm == LES_WARM_ZERO) {
        CK(cudaMemsetAsync(h->ph[h->cur], 0, h->n * sizeof(double), st));
        h->launches += launch_residual64<T>(g, h->ph[h->cur], (const T*)h->rhs, (T*)h->rr, h->vfluid, reducer(h),
                                            cond_args(h, RES_INIT, 0, 0), st);
    }
    if constexpr (std::is_same<T, float>::value) {
        if (h->warm == LES_WARM_NET && h->net && (h->net_start || h->net_every == 0)) {
            int rc = net_correct<T>(h, g, st);
            if (rc) return rc;
        }
    }
    if (h->net_async) CK(cudaMemsetAsync(&h->sc->qpend, 0, sizeof(int), st));   // no prediction pending yet
    h->rec_taken = false;
    if (h->record && h->rec_after == 0) record_start(h, st);
    CK(cudaGetLastError());
    return LES_OK;
}

template <typename T>
int solve_end(les_s* h, const Geo<T>& g, cudaStream_t st) {
    h->rec_valid = h->record && h->rec_taken;
    if (h->rec_valid) {
        h->launches += launch_record<T>(g, h->ph[h->cur], h->rec_p0, (T*)h->rec_delta, 0, st);
        CK(cudaGetLastError());
    }
    return LES_OK;
}

template <typename T>
void launch_refine(les_s* h, const Geo<T>& g, const CondArgs& ca, cudaStream_t st) {
    h->launches += launch_accum<T>(g, h->ph[h->cur], (const T*)h->dl[h->dcur], h->sc, ca.gate, st);
    h->launches += launch_residual64<T>(g, h->ph[h->cur], (const T*)h->rhs, (T*)h->rr, h->vfluid, reducer(h), ca, st);
}

bool est_pools(les_s* h, EstPool* pool);

// Host-driven loop.  After each batch of check_every sweeps the cheap
// estimate is read back; when it asks for it, the FP64 refinement runs and
// its true relative residual decides convergence.
template <typename T>
int sor_solve(les_s* h) {
    Geo<T> g = geo<T>(h);
    const les_grid_t& G = h->g;
    rec(h, 2);
    h->launches += launch_residual64<T>(g, h->ph[h->cur], (const T*)h->rhs, (T*)h->rr, h->vfluid, reducer(h),
                                        cond_args(h, RES_INIT, 0, 0), h->stream);
    rec(h, 3);
    CK(cudaGetLastError());
    if (h->timing) {
        CK(cudaEventSynchronize(h->ev[3]));
        h->tm.ms_residual += elapsed(h, 2, 3);
    }
    {
        rec(h, 2);
        int rs = solve_start<T>(h, g, h->stream);
        if (rs) return rs;
        rec(h, 3);
        if (h->timing && h->warm == LES_WARM_NET) {
            CK(cudaEventSynchronize(h->ev[3]));
            h->tm.ms_net += elapsed(h, 2, 3);
        }
    }
    int sweeps = 0, last_net = 0;
    bool fresh = true, conv = false;
    bool recorded = !h->record || h->rec_taken;
    const bool net_loop = std::is_same<T, float>::value && h->warm == LES_WARM_NET && h->net && h->net_every > 0;
    EstPool pool;
    const bool pooled = net_loop && est_pools(h, &pool);
    if (!G.fixed_sweeps && h->warm != LES_WARM_PREV) {
        // the start of the solve moved p: its residual may already pass the test
        int rc = fetch_scalars(h);
        if (rc) return rc;
        conv = h->sc_host->converged != 0;
    }
    while (sweeps < G.max_sweeps && !conv) {
        int n = G.fixed_sweeps ? G.max_sweeps
                               : (G.check_every < G.max_sweeps - sweeps ? G.check_every : G.max_sweeps - sweeps);
        if (net_loop && !G.fixed_sweeps) n = std::min(n, std::max(1, h->net_every - (sweeps - last_net)));
        rec(h, 2);
        long long nl = 0;
        run_sweeps<T>(h, g, n, fresh ? 1 : 0, nl, h->stream);
        h->launches += nl;
        rec(h, 3);
        sweeps += n;
        bool need = true;
        if (!G.fixed_sweeps) {
            h->launches += launch_estimate<T>(h, g, net_loop ? (T*)h->rcur : nullptr, cond_args(h, RES_LOOP, n, 0),
                                              h->stream, pooled ? &pool : nullptr);
            CK(cudaGetLastError());
            int rc = fetch_scalars(h);
            if (rc) return rc;
            need = h->sc_host->refine != 0;
        }
        rec(h, 4);
        if (h->timing) {
            CK(cudaEventSynchronize(h->ev[4]));
            h->tm.ms_sor += elapsed(h, 2, 3);
            h->tm.ms_residual += elapsed(h, 3, 4);
            h->tm.sor_sweeps += n;
            h->tm.sor_launches += nl;
        }
        fresh = false;
        const bool net_due = net_loop && sweeps - last_net >= h->net_every && sweeps < G.max_sweeps;
        const bool rec_due = !recorded && sweeps >= h->rec_after;
        if (need || rec_due) {
            rec(h, 3);
            launch_refine<T>(h, g, cond_args(h, G.fixed_sweeps ? RES_FIXED : RES_LOOP, n, 0), h->stream);
            rec(h, 4);
            CK(cudaGetLastError());
            int rc = fetch_scalars(h);
            if (rc) return rc;
            if (h->timing) h->tm.ms_residual += elapsed(h, 3, 4);
            fresh = true;
            conv = h->sc_host->converged != 0;
            if (conv || h->sc_host->nonfinite) break;
            if (rec_due) {
                record_start(h, h->stream);
                recorded = true;
            }
        }
        if constexpr (std::is_same<T, float>::value) {
            if (net_due) {
                last_net = sweeps;
                rec(h, 2);
                int rc = net_correct_loop<T>(h, g, h->stream, false, pooled);
                if (rc) return rc;
                rec(h, 3);
                if (h->timing) {
                    CK(cudaEventSynchronize(h->ev[3]));
                    h->tm.ms_net += elapsed(h, 2, 3);
                    h->tm.net_cycles += 1;
                }
                fresh = false;      // the correction now holds the network's step
            }
        }
    }
    h->sc_host->sweeps = sweeps;
    {
        int rs = solve_end<T>(h, g, h->stream);
        if (rs) return rs;
    }
    if (h->sc_host->timeout) return fail(h, LES_ETIMEOUT, "a bounded device wait (TMA tile load) timed out");
    if (h->sc_host->nonfinite) return fail(h, LES_ENONFINITE, "SOR residual is not finite");
    return (!G.fixed_sweeps && !conv) ? LES_ENOCONV : LES_OK;
}

// sweep configurations this handle can run: the plain tiles always, the TMA
// block tiles on FP32 grids, the persistent TMA tiles without periodic axes
bool tile_available(const les_s* h, int t) {
    if (t < 0 || t >= kNumSorTiles + kNumTmaTiles) return false;
    if (t < kNumSorTiles) return true;
    const int c = t - kNumSorTiles;
    return h->tma_ok && (c < kNumTmaBlockTiles || c >= kFirstMarchCfg || h->pipe_ok);
}

// Time `sweeps` sweeps per candidate (tile shape x k-chunk) on the current
// correction right-hand side; the sweeps touch only the scratch correction
// buffers, never the state.
template <typename T>
int autotune_impl(les_s* h, int sweeps, double* best_ms, int only_tile = -2, int only_kc = 0);

// time one configuration (the state is untouched; the current configuration is kept)
template <typename T>
int time_config_impl(les_s* h, int tile, int kc, int sweeps, double* ms) {
    const SorCfg keep = h->sor;
    int rc = autotune_impl<T>(h, sweeps, ms, tile, kc);
    h->sor = keep;
    return rc;
}

template <typename T>
int autotune_impl(les_s* h, int sweeps, double* best_ms, int only_tile, int only_kc) {
    Geo<T> g = geo<T>(h);
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    const int kcs[] = {4, 8, 16, 32, 0};
    int done_save = 0;
    CK(cudaMemcpyAsync(&done_save, &h->sc->done, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemsetAsync(&h->sc->done, 0, sizeof(int), h->stream));
    SorCfg keep = h->sor, best = keep;
    double bms = 1e300;
    for (int t = 0; t < kNumSorTiles + kNumTmaTiles; ++t)
        for (int kc : kcs) {
            if (!tile_available(h, t)) continue;
            if (kc > h->g.nz) continue;
            const bool march = t >= kNumSorTiles + kFirstMarchCfg && t < kNumSorTiles + kFirstColCfg;   // take kc
            if (((t >= kNumSorTiles && !march) || (t < kNumSorTiles && kSorTiles[t].tz > 0)) && kc != 0)
                continue;      // 3-D blocks ignore kc
            if (only_tile >= -1 && (t != only_tile || kc != only_kc)) continue;
            h->sor = SorCfg{t, kc};
            long long nl = 0;
            run_sweeps<T>(h, g, 2, 0, nl, h->stream);       // warm
            CK(cudaEventRecord(a, h->stream));
            run_sweeps<T>(h, g, sweeps, 0, nl, h->stream);
            CK(cudaEventRecord(b, h->stream));
            CK(cudaEventSynchronize(b));
            h->launches += nl;
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, a, b));
            double per = ms / sweeps;
            if (per < bms) {
                bms = per;
                best = h->sor;
            }
        }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    CK(cudaMemcpyAsync(&h->sc->done, &done_save, sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->sor = bms < 1e299 ? best : keep;
    h->graph_ok[0] = h->graph_ok[1] = false;
    if (best_ms) *best_ms = bms;
    return LES_OK;
}

template <typename T>
void launch_project_step(les_s* h, const Geo<T>& g, int cur, cudaStream_t st) {
    h->launches += launch_project<T>(g, (const T*)h->us, (const T*)h->vs, (const T*)h->ws, (T*)h->u, (T*)h->v,
                                     (T*)h->w, h->ph[cur], h->ph[1 - cur], h->sc, st);
}

// bondv1, les, velfg, adam, feedbf, bondv1 (outflow), rhs
template <typename T>
void launch_prefix(les_s* h, const Geo<T>& g, cudaStream_t s) {
    T* u = (T*)h->u;
    T* v = (T*)h->v;
    T* w = (T*)h->w;
    const InflowSeries ser{h->series_p, h->series_t, h->nseries, h->g.dt};
    h->launches += launch_bc<T>(g, u, v, w, h->inflow64, ser, h->g.turb, h->g.seed, h->sc, s);
    h->launches += launch_nut<T>(g, u, v, w, (T*)h->nut, s);
    h->launches += launch_momentum<T>(g, u, v, w, (const T*)h->nut, (T*)h->fu, (T*)h->fv, (T*)h->fw, (T*)h->us,
                                      (T*)h->vs, (T*)h->ws, h->sc, s);
    h->launches += launch_outflow<T>(g, u, (T*)h->us, (T*)h->vs, (T*)h->ws, reducer(h), s);
    h->launches += launch_rhs<T>(g, (const T*)h->us, (const T*)h->vs, (const T*)h->ws, (T*)h->rhs, h->vfluid,
                                 reducer(h), s);
}

// Host-driven step (used with phase timing and for les_pressure_solve).
template <typename T>
int step_host(les_s* h) {
    Geo<T> g = geo<T>(h);
    rec(h, 0);
    launch_prefix<T>(h, g, h->stream);
    rec(h, 1);
    CK(cudaGetLastError());
    int rc = sor_solve<T>(h);
    if (rc < 0) return rc;
    rec(h, 5);
    launch_project_step<T>(h, g, h->cur, h->stream);
    CK(cudaGetLastError());
    h->cur = 1 - h->cur;
    rec(h, 6);
    if (h->timing) {
        CK(cudaEventSynchronize(h->ev[6]));
        h->tm.ms_momentum += elapsed(h, 0, 1);
        h->tm.ms_project += elapsed(h, 5, 6);
        h->tm.steps += 1;
    }
    h->step += 1;
    return rc;
}

// Graph execution without device-side control flow.  A step launches the
// prefix kernels and the first FP64 residual, then replays a captured "chunk"
// of kChunkBatches batches (check_every sweeps, the estimate, a gated
// refinement).  Every kernel of a chunk returns at once when the device flag
// `done` is set, so the host can keep one chunk in flight and stop enqueueing
// when it sees the mapped copy of the flag: the GPU never waits for the host.
// With fixed_sweeps the whole step is one captured graph.
// the network correction runs inside the solve loop (FP32 grids)
bool net_in_loop(const les_s* h) {
    return h->prec == LES_FP32 && h->warm == LES_WARM_NET && h->net && h->net_every > 0;
}

// The estimate before each network correction inside the solve forms the
// network's pooled input (the TMA estimate, the in-place schedule, strides 4
// and 8): the correction then skips its pooling kernel and its re-read of
// the residual.  The overlapped schedule keeps the pooling on its own
// stream, since a prediction still running there reads the pooled input.
bool est_pools(les_s* h, EstPool* pool) {
    if (!net_in_loop(h) || !h->est_tma || h->net_async || h->net_own_pool || h->net_persistent) return false;
    return net_pool_target(h->net, h->d, pool);
}

constexpr int kChunkBatches = 10;
// with the network correction a batch is a whole cycle (sweeps, estimate,
// network, step): shorter chunks waste fewer done-gated launches after the
// stop test has passed
constexpr int kChunkCycles = 4;
int chunk_batches(const les_s* h) { return net_in_loop(h) ? kChunkCycles : kChunkBatches; }

template <typename T>
int capture_begin(les_s* h, cudaStream_t cs) {
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    return LES_OK;
}

template <typename T>
int capture_end(les_s* h, cudaStream_t cs, cudaGraphExec_t* out) {
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &gr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, LES_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    }
    if (*out) cudaGraphExecDestroy(*out);
    *out = nullptr;
    e = cudaGraphInstantiate(out, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return fail(h, LES_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    return LES_OK;
}


template <typename T>
int build_graph(les_s* h, int cur) {
    Geo<T> g = geo<T>(h);
    const les_grid_t& G = h->g;
    cudaStream_t cs = h->cap[0];
    const int save_cur = h->cur, save_dcur = h->dcur;
    const long long l0 = h->launches;
    h->cur = cur;
    h->dcur = 0;
    EstPool pool;
    bool pooled = false;
    if (net_in_loop(h)) {
        // allocate the network's workspace before the capture
        int rp = net_prepare(h->net, h->d, &h->net_gen);
        if (rp) {
            h->cur = save_cur;
            h->dcur = save_dcur;
            return fail(h, rp, "network workspace");
        }
        pooled = est_pools(h, &pool);
    }
    int rc = capture_begin<T>(h, cs);
    if (rc) return rc;
    long long nl = 0;
    if (G.fixed_sweeps) {
        launch_prefix<T>(h, g, cs);
        nl += launch_residual64<T>(g, h->ph[cur], (const T*)h->rhs, (T*)h->rr, h->vfluid, reducer(h),
                                   cond_args(h, RES_INIT, 0, 0), cs);
        run_sweeps<T>(h, g, G.max_sweeps, 1, nl, cs);
        launch_refine<T>(h, g, cond_args(h, RES_FIXED, G.max_sweeps, 0), cs);
        launch_project_step<T>(h, g, cur, cs);
        h->graph_launches[cur] = h->launches - l0 + nl;
    } else if (net_in_loop(h) && h->net_async && !h->record) {
        // the overlapped correction: each batch applies the prediction made
        // from the previous batch's residual (line search against the current
        // residual, which then becomes the residual of the corrected iterate)
        // and forks the next prediction onto the second stream, where it runs
        // during the next batch's sweeps; joined at the end of the chunk
        if constexpr (std::is_same<T, float>::value) {
            for (int b = 0; b < chunk_batches(h) && !rc; ++b) {
                run_sweeps<T>(h, g, h->net_every, 2, nl, cs);     // net_every even: d returns to dl[0]
                if (b > 0) CK(cudaStreamWaitEvent(cs, h->ev_pool, 0));      // the prediction has read rcur
                launch_estimate<T>(h, g, (T*)h->rcur, cond_args(h, RES_LOOP, h->net_every, 1), cs);
                launch_refine<T>(h, g, cond_args(h, RES_LOOP, h->net_every, 1), cs);
                if (b > 0) CK(cudaStreamWaitEvent(cs, h->ev_q, 0));         // the prediction is complete
                launch_warm_pending<T>(g, (T*)h->rcur, h->pred, (T*)h->dl[h->dcur], h->warm_scal + 1, reducer(h),
                                       cs);
                CK(cudaEventRecord(h->ev_fork, cs));
                CK(cudaStreamWaitEvent(h->s2, h->ev_fork, 0));
                rc = net_predict(h->net, h->d, (const float*)h->rcur, h->flags, h->pred, h->s2, &h->sc->done,
                                 h->ev_pool);
                if (rc) {
                    fail(h, rc, "network prediction failed");
                    break;
                }
                h->net_chunk_launches = net_launches(h->net);
                launch_set_flag(&h->sc->qpend, 1, &h->sc->done, h->s2);
                CK(cudaEventRecord(h->ev_q, h->s2));
            }
            cudaStreamWaitEvent(cs, h->ev_q, 0);                            // join
        }
    } else if (net_in_loop(h)) {
        // cycles of net_every sweeps, a forced refinement, the network
        // correction and the residual again, all gated on `done`
        if constexpr (std::is_same<T, float>::value) {
            for (int b = 0; b < chunk_batches(h); ++b) {
                run_sweeps<T>(h, g, h->net_every, 2, nl, cs);     // net_every even: d returns to dl[0]
                launch_estimate<T>(h, g, (T*)h->rcur, cond_args(h, RES_LOOP, h->net_every, 1), cs,
                                   pooled ? &pool : nullptr);
                launch_refine<T>(h, g, cond_args(h, RES_LOOP, h->net_every, 1), cs);
                rc = net_correct_loop<T>(h, g, cs, true, pooled);
                if (rc) break;
                h->net_chunk_launches = net_launches(h->net);
            }
        }
    } else {
        for (int b = 0; b < kChunkBatches; ++b) {
            run_sweeps<T>(h, g, G.check_every, 2, nl, cs);     // check_every even: d returns to dl[0]
            launch_estimate<T>(h, g, (T*)nullptr, cond_args(h, RES_LOOP, G.check_every, 1), cs);
            launch_refine<T>(h, g, cond_args(h, RES_LOOP, G.check_every, 1), cs);
        }
    }
    {
        const int rc2 = capture_end<T>(h, cs, &h->gexec[cur]);
        if (!rc) rc = rc2;
    }
    h->cur = save_cur;
    h->dcur = save_dcur;
    h->launches = l0;          // capture launches nothing
    if (rc) return rc;
    h->graph_ok[cur] = true;
    return LES_OK;
}

void fill_stats(les_s* h, les_stats_t* st, int status);

template <typename T>
int step_graph(les_s* h, int nsteps, les_stats_t* stats) {
    const les_grid_t& G = h->g;
    if (net_in_loop(h) && net_generation(h->net) != h->net_gen) h->graph_ok[0] = h->graph_ok[1] = false;
    for (int c = 0; c < 2; ++c)
        if (!h->graph_ok[c]) {
            int rc = build_graph<T>(h, c);
            if (rc) return rc;      // caller falls back to the host-driven loop
        }
    Geo<T> g = geo<T>(h);
    CK(cudaMemsetAsync(&h->sc->noconv_any, 0, sizeof(int), h->stream));
    const int per_chunk = chunk_batches(h) * (net_in_loop(h) ? h->net_every : G.check_every);
    const int max_chunks = (G.max_sweeps + per_chunk - 1) / per_chunk + 1;
    for (int s = 0; s < nsteps; ++s) {
        if (G.fixed_sweeps) {
            CK(cudaGraphLaunch(h->gexec[h->cur], h->stream));
            h->launches += h->graph_launches[h->cur];
        } else {
            *(volatile int*)h->done_host = 0;
            launch_prefix<T>(h, g, h->stream);
            h->launches += launch_residual64<T>(g, h->ph[h->cur], (const T*)h->rhs, (T*)h->rr, h->vfluid, reducer(h),
                                                cond_args(h, RES_INIT, 0, 0), h->stream);
            CK(cudaGetLastError());
            {
                int rs = solve_start<T>(h, g, h->stream);
                if (rs) return rs;
            }
            const long long per_batch = net_in_loop(h) ? h->net_every + 3 + h->net_chunk_launches + 2 +
                                                             (h->net_async && !h->record ? 1 : 0)
                                                       : G.check_every + 3;
            for (int c = 0; c < max_chunks; ++c) {
                CK(cudaGraphLaunch(h->gexec[h->cur], h->stream));
                CK(cudaEventRecord(h->chunk_ev[c & 1], h->stream));
                h->launches += chunk_batches(h) * per_batch;
                if (c >= 1) {
                    CK(cudaEventSynchronize(h->chunk_ev[(c - 1) & 1]));
                    if (*(volatile int*)h->done_host) break;
                }
            }
            {
                int rs = solve_end<T>(h, g, h->stream);
                if (rs) return rs;
            }
            launch_project_step<T>(h, g, h->cur, h->stream);
            CK(cudaGetLastError());
        }
        h->cur = 1 - h->cur;
        h->step += 1;
    }
    int rc = fetch_scalars(h);
    if (rc) return rc;
    int status = (!G.fixed_sweeps && h->sc_host->noconv_any) ? LES_ENOCONV : LES_OK;
    if (h->sc_host->timeout) return fail(h, LES_ETIMEOUT, "a bounded device wait (TMA tile load) timed out");
    if (h->sc_host->nonfinite) return fail(h, LES_ENONFINITE, "SOR residual is not finite");
    if (stats) fill_stats(h, stats, status);
    return status;
}

void fill_stats(les_s* h, les_stats_t* st, int status) {
    if (!st) return;
    const Scalars& s = *h->sc_host;
    st->sweeps = s.sweeps;
    st->status = status;
    st->rel_residual = s.rel;
    st->rhs_norm = std::sqrt(s.rhs2);
    st->rhs_mean = s.rhs_mean;
    st->mass_factor = s.mass_factor;
    st->q_in = s.q_in;
    st->q_out = s.q_out;
    st->p_mean = s.p_mean;
    st->step = h->step;
    st->launches = h->launches;
    st->graph = h->last_graph ? 1 : 0;
}

int validate(const les_grid_t* g) {
    if (!g) return fail(nullptr, LES_EINVAL, "grid is NULL");
    if (g->nx < 2 || g->ny < 2 || g->nz < 2) return fail(nullptr, LES_EINVAL, "nx, ny, nz must be >= 2");
    if ((long long)g->nx * g->ny * g->nz > (1LL << 31))
        return fail(nullptr, LES_EINVAL, "grid larger than 2^31 cells");
    if (g->bc_x != LES_BC_INOUT && g->bc_x != LES_BC_PERIODIC) return fail(nullptr, LES_EINVAL, "bad bc_x");
    if (g->bc_y != LES_BC_FREESLIP && g->bc_y != LES_BC_PERIODIC) return fail(nullptr, LES_EINVAL, "bad bc_y");
    if (g->bc_z != LES_BC_WALL && g->bc_z != LES_BC_PERIODIC) return fail(nullptr, LES_EINVAL, "bad bc_z");
    if ((g->bc_x == LES_BC_PERIODIC && g->nx % 2) || (g->bc_y == LES_BC_PERIODIC && g->ny % 2) ||
        (g->bc_z == LES_BC_PERIODIC && g->nz % 2))
        return fail(nullptr, LES_EINVAL, "a periodic axis needs an even cell count (red-black colouring)");
    if (!(g->dx > 0) || !(g->dy > 0) || !(g->dt > 0)) return fail(nullptr, LES_EINVAL, "dx, dy, dt must be > 0");
    if (!g->dz) return fail(nullptr, LES_EINVAL, "dz is NULL");
    for (int k = 0; k < g->nz; ++k)
        if (!(g->dz[k] > 0)) return fail(nullptr, LES_EINVAL, "dz[%d] must be > 0", k);
    if (!(g->omega > 0 && g->omega < 2)) return fail(nullptr, LES_EINVAL, "omega must be in (0, 2)");
    if (g->max_sweeps < 1 || g->check_every < 1) return fail(nullptr, LES_EINVAL, "max_sweeps, check_every >= 1");
    if (g->precision != LES_FP32 && g->precision != LES_FP64) return fail(nullptr, LES_EINVAL, "bad precision");
    if (!(g->cs >= 0) || !(g->nu >= 0) || !(g->turb >= 0) || !(g->tol >= 0))
        return fail(nullptr, LES_EINVAL, "cs, nu, turb, tol must be >= 0");
    return LES_OK;
}

template <typename T>
int init_tables(les_s* h) {
    const int nz = h->g.nz;
    std::vector<double> dzp(nz + 2), dzs(nz + 2), cT(nz + 2, 0.0), cB(nz + 2, 0.0), del(nz + 2, 0.0);
    for (int k = 1; k <= nz; ++k) dzp[k] = h->dz[k - 1];
    if (h->g.bc_z == LES_BC_PERIODIC) {
        dzp[0] = dzp[nz];
        dzp[nz + 1] = dzp[1];
    } else {
        dzp[0] = dzp[1];
        dzp[nz + 1] = dzp[nz];
    }
    for (int k = 0; k <= nz; ++k) dzs[k] = 0.5 * (dzp[k] + dzp[k + 1]);
    dzs[nz + 1] = dzp[nz + 1];
    for (int k = 1; k <= nz; ++k) {
        cT[k] = 1.0 / (dzp[k] * dzs[k]);
        cB[k] = 1.0 / (dzp[k] * dzs[k - 1]);
        double l = h->g.cs * std::cbrt(h->g.dx * h->g.dy * dzp[k]);
        del[k] = l * l;
    }
    std::vector<double> rdz(nz + 2), rdzs(nz + 2);
    for (int k = 0; k <= nz + 1; ++k) {
        rdz[k] = 1.0 / dzp[k];
        rdzs[k] = 1.0 / dzs[k];
    }
    int rc;
    if ((rc = upload_table<T>(h, h->krdz, rdz))) return rc;
    if ((rc = upload_table<T>(h, h->krdzs, rdzs))) return rc;
    if ((rc = upload_table<T>(h, h->kdz, dzp))) return rc;
    if ((rc = upload_table<T>(h, h->kdzs, dzs))) return rc;
    if ((rc = upload_table<T>(h, h->kcT, cT))) return rc;
    if ((rc = upload_table<T>(h, h->kcB, cB))) return rc;
    if ((rc = upload_table<T>(h, h->kdel, del))) return rc;
    if ((rc = upload_table<double>(h, h->dz64, dzp))) return rc;
    if ((rc = upload_table<double>(h, h->dzs64, dzs))) return rc;
    if ((rc = upload_table<double>(h, h->cT64, cT))) return rc;
    if ((rc = upload_table<double>(h, h->cB64, cB))) return rc;
    return LES_OK;
}

void release(les_s* h) {
    if (h->series_p) cudaFree(h->series_p);
    if (h->series_t) cudaFree(h->series_t);
    h->series_p = h->series_t = nullptr;
    for (cudaGraphExec_t& x : h->gexec)
        if (x) {
            cudaGraphExecDestroy(x);
            x = nullptr;
        }
    for (cudaStream_t& c : h->cap)
        if (c) {
            cudaStreamDestroy(c);
            c = nullptr;
        }
    for (cudaEvent_t& e : h->chunk_ev)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
    for (cudaEvent_t* e : {&h->ev_fork, &h->ev_pool, &h->ev_q})
        if (*e) {
            cudaEventDestroy(*e);
            *e = nullptr;
        }
    if (h->s2) cudaStreamSynchronize(h->s2), cudaStreamDestroy(h->s2);
    h->s2 = nullptr;
    if (h->done_host) cudaFreeHost(h->done_host);
    h->done_host = nullptr;
    for (cudaEvent_t& e : h->ev)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
    for (void* p : h->allocs) cudaFree(p);
    h->allocs.clear();
    if (h->sc_host) cudaFreeHost(h->sc_host);
    h->sc_host = nullptr;
}

int create_impl(les_s* h, const uint8_t* solid) {
    const les_grid_t& G = h->g;
    Dom& d = h->d;
    d.nx = G.nx;
    d.ny = G.ny;
    d.nz = G.nz;
    d.px = ((G.nx + 2 + OX) + 15) / 16 * 16;
    d.py = G.ny + 2;
    d.plane = (long long)d.px * d.py;
    d.perx = G.bc_x == LES_BC_PERIODIC;
    d.pery = G.bc_y == LES_BC_PERIODIC;
    d.perz = G.bc_z == LES_BC_PERIODIC;
    if (d.total() + 16 > 0x7fffffffLL) return fail(h, LES_EINVAL, "padded grid exceeds 2^31 elements");
    h->n = (size_t)d.total() + 16;     // slack so a vector load past the last row stays in bounds
    const size_t B = h->n * h->es;
    int rc;
    void** fields[] = {&h->u, &h->v, &h->w, &h->us, &h->vs, &h->ws, &h->fu, &h->fv, &h->fw,
                       &h->nut, &h->rhs, &h->tmp, &h->dl[0], &h->dl[1], &h->rr};
    for (void** f : fields)
        if ((rc = dalloc(h, f, B))) return rc;
    for (double*& f : h->ph)
        if ((rc = dalloc(h, (void**)&f, h->n * sizeof(double)))) return rc;
    if ((rc = dalloc(h, (void**)&h->flags, h->n))) return rc;
    const size_t nt = (size_t)G.nz + 2;
    void** tabs[] = {&h->kdz, &h->kdzs, &h->kcT, &h->kcB, &h->kdel, &h->krdz, &h->krdzs};
    for (void** t : tabs)
        if ((rc = dalloc(h, t, nt * h->es))) return rc;
    if ((rc = dalloc(h, (void**)&h->dz64, nt * sizeof(double)))) return rc;
    if ((rc = dalloc(h, (void**)&h->dzs64, nt * sizeof(double)))) return rc;
    if ((rc = dalloc(h, (void**)&h->cT64, nt * sizeof(double)))) return rc;
    if ((rc = dalloc(h, (void**)&h->cB64, nt * sizeof(double)))) return rc;
    if ((rc = dalloc(h, (void**)&h->inflow64, nt * sizeof(double)))) return rc;
    const int nb = max_reduce_blocks(d);
    if ((rc = dalloc(h, (void**)&h->partials, (size_t)3 * nb * sizeof(double)))) return rc;
    if ((rc = dalloc(h, (void**)&h->counter, sizeof(unsigned)))) return rc;
    if ((rc = dalloc(h, (void**)&h->sc, sizeof(Scalars)))) return rc;
    h->stage_elems = io_elems(h, 1) + io_elems(h, 2) + io_elems(h, 3) + io_elems(h, 0);
    if ((rc = dalloc(h, &h->stage, h->stage_elems * h->es))) return rc;
    for (cudaStream_t& c : h->cap) CK(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
    for (cudaEvent_t& e : h->chunk_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    if (cudaHostAlloc((void**)&h->done_host, sizeof(int), cudaHostAllocMapped) != cudaSuccess)
        return fail(h, LES_ENOMEM, "cudaHostAlloc failed");
    *h->done_host = 0;
    CK(cudaHostGetDevicePointer((void**)&h->done_dev, h->done_host, 0));
    if (cudaMallocHost((void**)&h->sc_host, sizeof(Scalars)) != cudaSuccess)
        return fail(h, LES_ENOMEM, "cudaMallocHost failed");
    memset(h->sc_host, 0, sizeof(Scalars));
    h->sc_host->mass_factor = 1.0;

    // obstacles: padded solid mask -> open-face flags (on the device)
    uint8_t* solid_d = nullptr;
    if ((rc = dalloc(h, (void**)&solid_d, h->n))) return rc;
    std::vector<uint8_t> tmp((size_t)G.nx * G.ny * G.nz);
    double vf = 0.0;
    for (int k = 0; k < G.nz; ++k)
        for (int j = 0; j < G.ny; ++j)
            for (int i = 0; i < G.nx; ++i) {
                size_t q = ((size_t)k * G.ny + j) * G.nx + i;
                tmp[q] = solid[q] ? 1 : 0;
                if (!tmp[q]) vf += h->dz[k];
            }
    h->vfluid = vf;
    uint8_t* st8 = (uint8_t*)h->stage;   // stage holds at least nx*ny*nz bytes
    CK(cudaMemcpyAsync(st8, tmp.data(), tmp.size(), cudaMemcpyHostToDevice, h->stream));
    {
        size_t n = tmp.size();
        k_unpack<uint8_t, uint8_t><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(d, st8, solid_d, 1, 1, 1, G.nx, G.ny, G.nz);
        k_flags<<<dim3((G.nx + 31) / 32, (G.ny + 7) / 8, G.nz), dim3(32, 8), 0, h->stream>>>(d, solid_d, h->flags);
        CK(cudaGetLastError());
    }
    CK(cudaMemcpyAsync(h->inflow64, h->inflow.data(), nt * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    rc = h->prec == LES_FP64 ? init_tables<double>(h) : init_tables<float>(h);
    if (rc) return rc;
    CK(h->prec == LES_FP64 ? sor_prepare<double>() : sor_prepare<float>());
    {
        unsigned long long* cnt = nullptr;
        if ((rc = dalloc(h, (void**)&cnt, sizeof(unsigned long long)))) return rc;
        launch_count_unknowns(d, h->flags, cnt, h->stream);
        unsigned long long hc = 0;
        CK(cudaMemcpyAsync(&hc, cnt, sizeof hc, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        h->n_unk = (double)hc;
    }
    if ((rc = dalloc(h, (void**)&h->diag64, (size_t)(G.nz + 2) * 64 * sizeof(double)))) return rc;
    if (h->prec == LES_FP32) launch_diag_table<float>(geo<float>(h), h->diag64, h->stream);
    else launch_diag_table<double>(geo<double>(h), h->diag64, h->stream);
    CK(cudaGetLastError());
    if (h->prec == LES_FP32) {
        // cn1 over (plane, open-face mask), read by the FP32 sweep kernels
        if ((rc = dalloc(h, (void**)&h->cn1tab, (size_t)(G.nz + 2) * 64 * sizeof(float)))) return rc;
        launch_cn1_table(geo<float>(h), h->cn1tab, h->stream);
        CK(cudaGetLastError());
        if ((rc = dalloc(h, (void**)&h->coltab, (size_t)(G.nz + 2 + kColTableRows) * 68 * sizeof(float)))) return rc;
        launch_col_table(geo<float>(h), h->cn1tab, h->coltab, h->stream);
        CK(cudaGetLastError());
        if (tma_supported(d)) {
            CK(tma_prepare());
            h->tma_ok = tma_encode(d, (float*)h->dl[0], (float*)h->dl[1], (float*)h->rr, h->flags, h->tma);
            h->pipe_ok = h->tma_ok && pipe_supported(d);
            h->est_tma = h->tma_ok && !d.perx && !d.pery && !d.perz &&
                         tma_encode_est(d, (float*)h->dl[0], (float*)h->dl[1], (float*)h->rr, h->flags, h->est_maps);
        }
        CK(cudaStreamSynchronize(h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    return LES_OK;
}

template <typename T>
int set_fields_impl(les_s* h, const void* u, const void* v, const void* w, const void* p) {
    int rc;
    size_t off = 0;
    if (u && (rc = upload<T>(h, h->u, 1, u, off))) return rc;
    off += io_elems(h, 1);
    if (v && (rc = upload<T>(h, h->v, 2, v, off))) return rc;
    off += io_elems(h, 2);
    if (w && (rc = upload<T>(h, h->w, 3, w, off))) return rc;
    off += io_elems(h, 3);
    if (p && (rc = upload<T, double>(h, h->ph[h->cur], 0, p, off))) return rc;
    return LES_OK;
}

template <typename T>
int get_fields_impl(les_s* h, void* u, void* v, void* w, void* p) {
    int rc;
    size_t off = 0;
    if (u && (rc = download<T>(h, h->u, 1, u, off))) return rc;
    off += io_elems(h, 1);
    if (v && (rc = download<T>(h, h->v, 2, v, off))) return rc;
    off += io_elems(h, 2);
    if (w && (rc = download<T>(h, h->w, 3, w, off))) return rc;
    off += io_elems(h, 3);
    if (p && (rc = download<T, double>(h, h->ph[h->cur], 0, p, off))) return rc;
    CK(cudaStreamSynchronize(h->stream));
    return LES_OK;
}

template <typename T>
int get_aux_impl(les_s* h, int which, void* out) {
    const void* src = nullptr;
    int stag = 0;
    switch (which) {
        case LES_AUX_NUT: src = h->nut; break;
        case LES_AUX_RHS: {
            Geo<T> g = geo<T>(h);
            h->launches += launch_rhs_eff<T>(g, (const T*)h->rhs, (T*)h->tmp, h->sc, h->stream);
            CK(cudaGetLastError());
            src = h->tmp;
            break;
        }
        case LES_AUX_USTAR: src = h->us; stag = 1; break;
        case LES_AUX_VSTAR: src = h->vs; stag = 2; break;
        case LES_AUX_WSTAR: src = h->ws; stag = 3; break;
        case LES_AUX_FU: src = h->fu; stag = 1; break;
        case LES_AUX_FV: src = h->fv; stag = 2; break;
        case LES_AUX_FW: src = h->fw; stag = 3; break;
        case LES_AUX_R0:
        case LES_AUX_DELTA:
            if (!h->record) return fail(h, LES_EINVAL, "recording is off (les_set_record)");
            if (!h->rec_valid)
                return fail(h, LES_ESTATE, "the last solve recorded no pair (it ended before the record point)");
            src = which == LES_AUX_R0 ? h->rec_r0 : h->rec_delta;
            break;
        case LES_AUX_NET_IN:
        case LES_AUX_NET_Q:
            if (!h->record) return fail(h, LES_EINVAL, "recording is off (les_set_record)");
            if (!h->net_taken) return fail(h, LES_ESTATE, "no start-of-solve network prediction recorded yet");
            if (which == LES_AUX_NET_Q) {
                CK(cudaMemcpyAsync(out, h->rec_netq, (size_t)h->g.nx * h->g.ny * h->g.nz * sizeof(float),
                                   cudaMemcpyDeviceToHost, h->stream));
                CK(cudaStreamSynchronize(h->stream));
                return LES_OK;
            }
            src = h->rec_netin;
            break;
        case LES_AUX_MASK: {
            Geo<T> g = geo<T>(h);
            h->launches += launch_record<T>(g, nullptr, nullptr, (T*)h->tmp, 1, h->stream);
            CK(cudaGetLastError());
            src = h->tmp;
            break;
        }
        default: return fail(h, LES_EINVAL, "unknown aux array %d", which);
    }
    int rc = download<T>(h, src, stag, out, 0);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream));
    return LES_OK;
}

template <typename T>
int pressure_solve_impl(les_s* h, const void* rhs, les_stats_t* st) {
    Geo<T> g = geo<T>(h);
    if (rhs) {
        int rc = upload<T>(h, h->rhs, 0, rhs, 0);
        if (rc) return rc;
        h->launches += launch_rhs_mean<T>(g, (T*)h->rhs, h->vfluid, reducer(h), h->stream);
        CK(cudaGetLastError());
    }
    int rc = sor_solve<T>(h);
    if (rc < 0) return rc;
    // gauge: p_out = p - mean (velocities untouched)
    h->launches += launch_gauge<T>(g, h->ph[h->cur], h->ph[1 - h->cur], h->sc, h->stream);
    CK(cudaGetLastError());
    h->cur = 1 - h->cur;
    CK(cudaStreamSynchronize(h->stream));
    fill_stats(h, st, rc);
    return rc;
}

// les_sor_compare: sweeps of one variant on A d = rhs - A p0 from d = 0 on
// the scratch correction buffers (the solver's residual buffer holds r; both
// are re-formed at the next solve), p0 + d and its FP64 residual
template <typename T>
int sor_compare_impl(les_s* h, int variant, double omega, int sweeps, const double* rhs, const double* p0,
                     double* p_out, double* ms_per_sweep, double* rel_residual) {
    Geo<T> g = geo<T>(h);
    if (omega > 0.0) g.omega = (T)omega;
    const size_t nbytes = h->n * sizeof(double);
    int rc;
    if (!h->cmp_p0) {
        if ((rc = dalloc(h, (void**)&h->cmp_p0, nbytes)) || (rc = dalloc(h, (void**)&h->cmp_b, nbytes)) ||
            (rc = dalloc(h, (void**)&h->cmp_pn, nbytes)) || (rc = dalloc(h, (void**)&h->cmp_out, 4 * sizeof(double))))
            return rc;
        CK(cudaMemsetAsync(h->cmp_p0, 0, nbytes, h->stream));
        CK(cudaMemsetAsync(h->cmp_b, 0, nbytes, h->stream));
    }
    if (variant == LES_SOR_TWINNED && !h->twin && (rc = dalloc(h, &h->twin, 2 * h->n * h->es))) return rc;
    if ((rc = upload<double, double>(h, h->cmp_p0, 0, p0, 0))) return rc;
    if ((rc = upload<double, double>(h, h->cmp_b, 0, rhs, 0))) return rc;
    const Reduce red{h->partials, h->counter, h->sc};
    h->launches += launch_cmp_residual<T>(g, h->cmp_p0, h->cmp_b, (T*)h->rr, red, h->cmp_out, h->stream);
    // the sweep kernels return at once once a solve is done: clear the flag for
    // the call and put it back afterwards
    int done_save = 0;
    CK(cudaMemcpyAsync(&done_save, &h->sc->done, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemsetAsync(&h->sc->done, 0, sizeof(int), h->stream));
    const int dcur_save = h->dcur;
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    CK(cudaEventRecord(a, h->stream));
    long long nl = 0;
    const T* dres;
    int stride;
    if (variant == LES_SOR_REDBLACK) {
        const int dc = run_sweeps<T>(h, g, sweeps, 1, nl, h->stream);
        dres = (const T*)h->dl[dc];
        stride = 1;
    } else {
        CK(cudaMemsetAsync(h->twin, 0, 2 * h->n * h->es, h->stream));
        for (int sw = 0; sw < sweeps; ++sw) {
            nl += launch_twin_half<T>(g, h->twin, (const T*)h->rr, 0, g.omega, h->stream);
            nl += launch_twin_half<T>(g, h->twin, (const T*)h->rr, 1, g.omega, h->stream);
        }
        dres = (const T*)h->twin;      // copy 0 holds the iterate after a whole sweep
        stride = 2;
    }
    CK(cudaEventRecord(b, h->stream));
    h->launches += nl;
    h->launches += launch_cmp_add<T>(g, h->cmp_p0, dres, stride, h->cmp_pn, h->n, h->stream);
    h->launches += launch_cmp_residual<T>(g, h->cmp_pn, h->cmp_b, (T*)h->rr, red, h->cmp_out + 2, h->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&h->sc->done, &done_save, sizeof(int), cudaMemcpyHostToDevice, h->stream));
    double norms[4];
    CK(cudaMemcpyAsync(norms, h->cmp_out, sizeof norms, cudaMemcpyDeviceToHost, h->stream));
    if (p_out && (rc = download<double, double>(h, h->cmp_pn, 0, p_out, 0))) return rc;
    CK(cudaStreamSynchronize(h->stream));
    h->dcur = dcur_save;
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ms_per_sweep = ms / sweeps;
    *rel_residual = norms[3] > 0.0 ? std::sqrt(norms[2] / norms[3]) : std::sqrt(norms[2]);
    return LES_OK;
}

// checkpoint blob: header, then the raw padded arrays and the inflow
struct StateHeader {
    uint64_t magic;
    int32_t nx, ny, nz, prec;
    int64_t step;
    double turb;
    uint64_t seed;
    uint64_t n, es;
};
constexpr uint64_t kMagic = 0x4c45534742333030ull;  // "LESGB300"

size_t state_size(const les_s* h) {
    return sizeof(StateHeader) + 6 * h->n * h->es + h->n * sizeof(double) + h->inflow.size() * sizeof(double);
}

}  // namespace

// ===========================================================================
// extern "C" entry points

extern "C" {

const char* les_version(void) { return kVersion; }

int les_selftest_wait_timeout(int64_t limit_ns, void* stream) {
    if (limit_ns < 1000 || limit_ns > 2000000000LL) return fail(nullptr, LES_EINVAL, "limit_ns must be 1e3..2e9");
    int* d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return fail(nullptr, LES_ENOMEM, "self-test flag");
    cudaStream_t s = (cudaStream_t)stream;
    int host = -1;
    launch_wait_selftest((unsigned long long)limit_ns, d, s);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host, d, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return fail(nullptr, LES_ECUDA, "wait self-test: %s", cudaGetErrorString(e));
    if (host == 1) return fail(nullptr, LES_ETIMEOUT, "bounded wait gave up after %lld ns (expected)",
                               (long long)limit_ns);
    return LES_OK;
}

int les_profiler_range(int32_t start) {
    cudaError_t e = start ? cudaProfilerStart() : cudaProfilerStop();
    return e == cudaSuccess ? LES_OK : fail(nullptr, LES_ECUDA, "profiler range: %s", cudaGetErrorString(e));
}

const char* les_last_error(les_handle h) { return h ? h->err : g_static_err; }

int les_create(const les_grid_t* grid, const uint8_t* solid, const double* inflow_u, void* stream,
               les_handle* out) {
    if (!out) return fail(nullptr, LES_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate(grid);
    if (rc) return rc;
    if (!solid) return fail(nullptr, LES_EINVAL, "solid is NULL");
    if (!inflow_u && grid->bc_x == LES_BC_INOUT) return fail(nullptr, LES_EINVAL, "inflow_u is NULL");
    les_s* h = new (std::nothrow) les_s();
    if (!h) return fail(nullptr, LES_ENOMEM, "out of host memory");
    h->g = *grid;
    h->dz.assign(grid->dz, grid->dz + grid->nz);
    h->g.dz = nullptr;
    h->prec = grid->precision;
    h->es = h->prec == LES_FP64 ? sizeof(double) : sizeof(float);
    h->stream = (cudaStream_t)stream;
    h->inflow.assign((size_t)grid->nz + 2, 0.0);
    if (inflow_u)
        for (int k = 1; k <= grid->nz; ++k) h->inflow[k] = inflow_u[k - 1];
    rc = create_impl(h, solid);
    if (rc) {
        snprintf(g_static_err, sizeof g_static_err, "%s", h->err);
        release(h);
        delete h;
        return rc;
    }
    *out = h;
    return LES_OK;
}

void les_destroy(les_handle h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    release(h);
    delete h;
}

int les_set_fields(les_handle h, const void* u, const void* v, const void* w, const void* p) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    return h->prec == LES_FP64 ? set_fields_impl<double>(h, u, v, w, p) : set_fields_impl<float>(h, u, v, w, p);
}

int les_get_fields(les_handle h, void* u, void* v, void* w, void* p) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    return h->prec == LES_FP64 ? get_fields_impl<double>(h, u, v, w, p) : get_fields_impl<float>(h, u, v, w, p);
}

int les_set_inflow(les_handle h, const double* inflow_u, double turb, uint64_t seed) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    if (!inflow_u) return fail(h, LES_EINVAL, "inflow_u is NULL");
    if (!(turb >= 0)) return fail(h, LES_EINVAL, "turb must be >= 0");
    for (int k = 1; k <= h->g.nz; ++k) h->inflow[k] = inflow_u[k - 1];
    h->g.turb = turb;
    h->g.seed = seed;
    CK(cudaMemcpyAsync(h->inflow64, h->inflow.data(), h->inflow.size() * sizeof(double), cudaMemcpyHostToDevice,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LES_OK;
}

int les_set_inflow_series(les_handle h, int32_t n, const double* times, const double* profiles) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    if (n < 0 || (n > 0 && (!times || !profiles))) return fail(h, LES_EINVAL, "bad inflow series");
    for (int m = 1; m < n; ++m)
        if (!(times[m] > times[m - 1])) return fail(h, LES_EINVAL, "inflow series times must increase");
    CK(cudaStreamSynchronize(h->stream));
    const int sk = h->g.nz + 2;
    if (n > h->series_cap) {
        if (h->series_p) cudaFree(h->series_p);
        if (h->series_t) cudaFree(h->series_t);
        h->series_p = h->series_t = nullptr;
        h->series_cap = 0;
        if (cudaMalloc(&h->series_p, (size_t)n * sk * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&h->series_t, (size_t)n * sizeof(double)) != cudaSuccess)
            return fail(h, LES_ENOMEM, "inflow series");
        h->series_cap = n;
    }
    if (n > 0) {
        std::vector<double> p((size_t)n * sk, 0.0);
        for (int m = 0; m < n; ++m)
            for (int k = 1; k <= h->g.nz; ++k) p[(size_t)m * sk + k] = profiles[(size_t)m * h->g.nz + k - 1];
        CK(cudaMemcpy(h->series_p, p.data(), p.size() * sizeof(double), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->series_t, times, (size_t)n * sizeof(double), cudaMemcpyHostToDevice));
    }
    h->nseries = n;
    h->graph_ok[0] = h->graph_ok[1] = false;      // a fixed-sweep graph holds the bondv1 arguments
    return LES_OK;
}

int les_step(les_handle h, int32_t nsteps, les_stats_t* stats) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    if (nsteps < 0) return fail(h, LES_EINVAL, "nsteps < 0");
    if (nsteps == 0) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return fail(h, LES_ECUDA, "step: %s", cudaGetErrorString(e));
        fill_stats(h, stats, LES_OK);
        return LES_OK;
    }
    // chunk graphs need an even batch (the ping-pong returns to the same buffer)
    // and a sweep budget made of whole batches; otherwise the host loop runs
    // (a fixed-sweep graph captures the whole step, so it runs without the
    // warm-start network and the recording; those use the chunked path)
    // network corrections inside a solve and recording after the start run
    // from the host loop
    const bool extras = h->record || h->warm != LES_WARM_PREV;
    const bool host_only = h->record && h->rec_after > 0;
    const int cycle = net_in_loop(h) ? h->net_every : h->g.check_every;
    const bool graph_ok = h->use_graph && !h->timing && !host_only &&
                          ((h->g.fixed_sweeps && !extras) ||
                           (!h->g.fixed_sweeps && cycle % 2 == 0 && h->g.max_sweeps % cycle == 0));
    h->last_graph = graph_ok;
    if (graph_ok) {
        int rc = h->prec == LES_FP64 ? step_graph<double>(h, nsteps, stats) : step_graph<float>(h, nsteps, stats);
        if (rc != LES_ECUDA || h->graph_ok[0] && h->graph_ok[1]) return rc;
        // the graph could not be built on this driver: keep the message, run
        // the same kernels from the host-driven loop from now on
        h->use_graph = false;
        h->graph_failed = true;
        h->last_graph = false;
    }
    int worst = LES_OK;
    for (int s = 0; s < nsteps; ++s) {
        int rc = h->prec == LES_FP64 ? step_host<double>(h) : step_host<float>(h);
        if (rc < 0) return rc;
        if (rc == LES_ENOCONV) worst = LES_ENOCONV;
        if (stats && s == nsteps - 1) {
            cudaError_t e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) return fail(h, LES_ECUDA, "step: %s", cudaGetErrorString(e));
            fill_stats(h, stats, rc);
        }
    }
    return worst;
}

int les_pressure_solve(les_handle h, const void* rhs, les_stats_t* stats) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    return h->prec == LES_FP64 ? pressure_solve_impl<double>(h, rhs, stats)
                               : pressure_solve_impl<float>(h, rhs, stats);
}

int les_get_aux(les_handle h, int32_t which, void* out) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    if (!out) return fail(h, LES_EINVAL, "out is NULL");
    return h->prec == LES_FP64 ? get_aux_impl<double>(h, which, out) : get_aux_impl<float>(h, which, out);
}

int les_get_state(les_handle h, void* buf, size_t* len) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    if (!len) return fail(h, LES_EINVAL, "len is NULL");
    size_t need = state_size(h);
    if (!buf) {
        *len = need;
        return LES_OK;
    }
    if (*len < need) return fail(h, LES_EINVAL, "state buffer too small (%zu < %zu)", *len, need);
    StateHeader hd{kMagic, h->g.nx, h->g.ny, h->g.nz, h->prec, h->step, h->g.turb, h->g.seed, h->n, h->es};
    char* b = (char*)buf;
    memcpy(b, &hd, sizeof hd);
    b += sizeof hd;
    const void* arrs[] = {h->u, h->v, h->w, h->fu, h->fv, h->fw, h->ph[h->cur]};
    for (int a = 0; a < 7; ++a) {
        const size_t B = h->n * (a == 6 ? sizeof(double) : h->es);
        CK(cudaMemcpyAsync(b, arrs[a], B, cudaMemcpyDeviceToHost, h->stream));
        b += B;
    }
    CK(cudaStreamSynchronize(h->stream));
    memcpy(b, h->inflow.data(), h->inflow.size() * sizeof(double));
    *len = need;
    return LES_OK;
}

int les_set_state(les_handle h, const void* buf, size_t len) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    if (!buf || len < sizeof(StateHeader)) return fail(h, LES_ESTATE, "state blob too small");
    StateHeader hd;
    memcpy(&hd, buf, sizeof hd);
    if (hd.magic != kMagic || hd.nx != h->g.nx || hd.ny != h->g.ny || hd.nz != h->g.nz || hd.prec != h->prec ||
        hd.n != h->n || hd.es != h->es || len != state_size(h))
        return fail(h, LES_ESTATE, "state blob does not match this handle");
    const char* b = (const char*)buf + sizeof hd;
    void* arrs[] = {h->u, h->v, h->w, h->fu, h->fv, h->fw, h->ph[h->cur]};
    for (int a = 0; a < 7; ++a) {
        const size_t B = h->n * (a == 6 ? sizeof(double) : h->es);
        CK(cudaMemcpyAsync(arrs[a], b, B, cudaMemcpyHostToDevice, h->stream));
        b += B;
    }
    memcpy(h->inflow.data(), b, h->inflow.size() * sizeof(double));
    CK(cudaMemcpyAsync(h->inflow64, h->inflow.data(), h->inflow.size() * sizeof(double), cudaMemcpyHostToDevice,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->step = hd.step;
    h->g.turb = hd.turb;
    h->g.seed = hd.seed;
    long long st = hd.step;
    CK(cudaMemcpyAsync(&h->sc->step, &st, sizeof st, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LES_OK;
}

int les_set_sor_config(les_handle h, int32_t tile, int32_t kc) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    if (tile < -1 || tile >= kNumSorTiles + kNumTmaTiles) return fail(h, LES_EINVAL, "tile %d out of range", tile);
    if (tile >= 0 && !tile_available(h, tile))
        return fail(h, LES_EINVAL, "tile %d needs an FP32 grid (persistent TMA tiles: no periodic axis)", tile);
    h->sor = SorCfg{tile, kc};
    h->graph_ok[0] = h->graph_ok[1] = false;
    return LES_OK;
}

int les_set_graph(les_handle h, int32_t enable) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    h->use_graph = enable != 0;
    return LES_OK;
}

int les_get_sor_config(les_handle h, int32_t* tile, int32_t* kc) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    if (tile) *tile = h->sor.tile;
    if (kc) *kc = h->sor.kc;
    return LES_OK;
}

int les_sor_tile(int32_t tile, int32_t* tx, int32_t* ty, int32_t* tz) {
    if (tile >= kNumSorTiles && tile < kNumSorTiles + kNumTmaTiles) {
        const int c = tile - kNumSorTiles;
        const bool march = c >= kFirstMarchCfg && c < kFirstColCfg;   // k-marching column: tz = 0
        if (tx) *tx = march ? 30 : 28;
        if (ty) *ty = kTmaCfg[c][0];
        if (tz) *tz = march ? 0 : kTmaCfg[c][1];
        return LES_OK;
    }
    if (tile < 0 || tile >= kNumSorTiles) return fail(nullptr, LES_EINVAL, "tile %d out of range", tile);
    if (tx) *tx = kSorTiles[tile].tx;
    if (ty) *ty = kSorTiles[tile].ty;
    if (tz) *tz = kSorTiles[tile].tz;
    return LES_OK;
}

int les_sor_compare(les_handle h, int32_t variant, double omega, int32_t sweeps, const double* rhs,
                    const double* p0, double* p_out, double* ms_per_sweep, double* rel_residual) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    if (variant != LES_SOR_REDBLACK && variant != LES_SOR_TWINNED)
        return fail(h, LES_EINVAL, "variant %d is not LES_SOR_REDBLACK or LES_SOR_TWINNED", variant);
    if (sweeps < 1) return fail(h, LES_EINVAL, "sweeps must be >= 1");
    if (!rhs || !p0 || !ms_per_sweep || !rel_residual)
        return fail(h, LES_EINVAL, "rhs, p0, ms_per_sweep and rel_residual must be set");
    return h->prec == LES_FP64
               ? sor_compare_impl<double>(h, variant, omega, sweeps, rhs, p0, p_out, ms_per_sweep, rel_residual)
               : sor_compare_impl<float>(h, variant, omega, sweeps, rhs, p0, p_out, ms_per_sweep, rel_residual);
}

int les_time_sor(les_handle h, int32_t tile, int32_t kc, int32_t sweeps, double* ms_per_sweep) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    if (sweeps < 1 || !ms_per_sweep) return fail(h, LES_EINVAL, "sweeps must be >= 1 and ms_per_sweep set");
    if (!tile_available(h, tile)) return fail(h, LES_EINVAL, "tile %d not available on this grid", tile);
    *ms_per_sweep = -1.0;
    int rc = h->prec == LES_FP64 ? time_config_impl<double>(h, tile, kc, sweeps, ms_per_sweep)
                                 : time_config_impl<float>(h, tile, kc, sweeps, ms_per_sweep);
    if (!rc && *ms_per_sweep > 1e299) return fail(h, LES_EINVAL, "configuration (%d, %d) not valid", tile, kc);
    return rc;
}

int les_autotune_sor(les_handle h, int32_t sweeps, double* best_ms_per_sweep) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    if (sweeps < 1) return fail(h, LES_EINVAL, "sweeps must be >= 1");
    return h->prec == LES_FP64 ? autotune_impl<double>(h, sweeps, best_ms_per_sweep)
                               : autotune_impl<float>(h, sweeps, best_ms_per_sweep);
}

int les_set_warmstart(les_handle h, int32_t mode, les_net net) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    if (mode == LES_WARM_PREV || mode == LES_WARM_ZERO) {
        h->warm = mode;
        h->net = nullptr;
        h->graph_ok[0] = h->graph_ok[1] = false;
        return LES_OK;
    }
    if (mode != LES_WARM_NET || !net) return fail(h, LES_EINVAL, "bad warm-start mode or NULL network");
    if (h->prec != LES_FP32) return fail(h, LES_EINVAL, "the learned warm start runs on FP32 grids");
    if (!h->pred) {
        int rc = dalloc(h, (void**)&h->pred, (size_t)h->g.nx * h->g.ny * h->g.nz * sizeof(float));
        if (rc) return rc;
        if ((rc = dalloc(h, (void**)&h->warm_scal, 4 * sizeof(double)))) return rc;
        if ((rc = dalloc(h, &h->rcur, h->n * h->es))) return rc;
    }
    h->warm = LES_WARM_NET;
    h->net = net;
    h->graph_ok[0] = h->graph_ok[1] = false;
    return LES_OK;
}

int les_set_net_start(les_handle h, int32_t enable) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    h->net_start = enable != 0;
    return LES_OK;
}

int les_set_net_async(les_handle h, int32_t enable) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    if (enable && !h->s2) {
        CK(cudaStreamCreateWithFlags(&h->s2, cudaStreamNonBlocking));
        for (cudaEvent_t* e : {&h->ev_fork, &h->ev_pool, &h->ev_q})
            CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
    h->net_async = enable != 0;
    h->graph_ok[0] = h->graph_ok[1] = false;
    return LES_OK;
}

int les_set_net_kernels(les_handle h, int32_t mode) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    const int layout = mode & ~LES_NET_KERNELS_OWN_POOL;
    if (layout < LES_NET_KERNELS_FOLDED || layout > LES_NET_KERNELS_LAYERS)
        return fail(h, LES_EINVAL, "network kernel layout must be 0, 1 or 2, optionally with LES_NET_KERNELS_OWN_POOL");
    h->net_kernels = layout;
    h->net_own_pool = (mode & LES_NET_KERNELS_OWN_POOL) != 0;
    h->net_persistent = layout == LES_NET_KERNELS_PERSISTENT;
    h->graph_ok[0] = h->graph_ok[1] = false;
    return LES_OK;
}

int les_set_net_schedule(les_handle h, int32_t every_sweeps) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    if (every_sweeps < 0) return fail(h, LES_EINVAL, "every_sweeps must be >= 0");
    h->net_every = every_sweeps;
    h->graph_ok[0] = h->graph_ok[1] = false;
    return LES_OK;
}

int les_set_record_at(les_handle h, int32_t after_sweeps) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    if (after_sweeps < 0) return fail(h, LES_EINVAL, "after_sweeps must be >= 0");
    h->rec_after = after_sweeps;
    return LES_OK;
}

int les_set_record(les_handle h, int32_t enable) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    h->graph_ok[0] = h->graph_ok[1] = false;      // the overlapped loop is captured without recording
    if (enable && !h->rec_p0) {
        int rc = dalloc(h, (void**)&h->rec_p0, h->n * sizeof(double));
        if (rc) return rc;
        if ((rc = dalloc(h, &h->rec_r0, h->n * h->es))) return rc;
        if ((rc = dalloc(h, &h->rec_delta, h->n * h->es))) return rc;
        if ((rc = dalloc(h, &h->rec_netin, h->n * h->es))) return rc;
        if ((rc = dalloc(h, (void**)&h->rec_netq, (size_t)h->g.nx * h->g.ny * h->g.nz * sizeof(float)))) return rc;
    }
    h->record = enable != 0;
    return LES_OK;
}

int les_set_timing(les_handle h, int32_t enable) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    if (enable && !h->ev[0])
        for (cudaEvent_t& e : h->ev) CK(cudaEventCreate(&e));
    h->timing = enable != 0;
    h->tm = les_timing_t{};
    return LES_OK;
}

int les_get_timing(les_handle h, les_timing_t* t) {
    if (!h) return fail(nullptr, LES_EINVAL, "handle is NULL");
    if (!t) return fail(h, LES_EINVAL, "t is NULL");
    *t = h->tm;
    t->launches = h->launches;
    return LES_OK;
}

}  // extern "C"

// ===========================================================================
// ensemble support: a member is an ordinary FP32 domain handle
namespace les {

int member_check(les_s* h, char* why, size_t n) {
    if (!h) {
        snprintf(why, n, "member handle is NULL");
        return LES_EINVAL;
    }
    if (h->prec != LES_FP32) {
        snprintf(why, n, "ensemble members run in FP32");
        return LES_EINVAL;
    }
    return LES_OK;
}

void member_fill(les_s* h, EnsMember<float>& M, int ens_tile, int parity) {
    const Dom& d = h->d;
    M.g = geo<float>(h);
    M.dl[0] = (float*)h->dl[0];
    M.dl[1] = (float*)h->dl[1];
    M.rr = (float*)h->rr;
    M.rhs = (const float*)h->rhs;
    M.ph = h->ph[parity];
    M.vfluid = h->vfluid;
    M.tol = h->g.tol;
    M.limit = h->g.max_sweeps;
    M.red = reducer(h);
    const SorTile t = ens_tile_shape(ens_tile);
    M.sgrid[0] = (d.nx + t.tx - 1) / t.tx;
    M.sgrid[1] = (d.ny + t.ty - 1) / t.ty;
    M.sgrid[2] = (d.nz + t.tz - 1) / t.tz;
    M.egrid[0] = (d.nx + 31) / 32;
    M.egrid[1] = (d.ny + 7) / 8;
    M.egrid[2] = (d.nz + kEstChunk - 1) / kEstChunk;
    M.agrid[0] = (d.nx + 31) / 32;
    M.agrid[1] = (d.ny + 7) / 8;
    M.agrid[2] = d.nz;
    M.rblocks = reduce_blocks(d);
    M.rcur = net_in_loop(h) ? (float*)h->rcur : nullptr;
}

int member_check_every(const les_s* h) { return h->g.check_every; }
int member_max_sweeps(const les_s* h) { return h->g.max_sweeps; }
cudaStream_t member_stream(const les_s* h) { return h->stream; }

int member_prefix(les_s* h, cudaStream_t s) {
    Geo<float> g = geo<float>(h);
    const long long l0 = h->launches;
    launch_prefix<float>(h, g, s);
    CK(cudaGetLastError());
    return (int)(h->launches - l0);
}

int member_finish(les_s* h, cudaStream_t s) {
    Geo<float> g = geo<float>(h);
    launch_project_step<float>(h, g, h->cur, s);
    CK(cudaGetLastError());
    h->cur = 1 - h->cur;
    h->step += 1;
    return LES_OK;
}

int member_stats(les_s* h, les_stats_t* st) {
    int rc = fetch_scalars(h);
    if (rc) return rc;
    int status = (!h->g.fixed_sweeps && h->sc_host->noconv_any) ? LES_ENOCONV : LES_OK;
    if (h->sc_host->nonfinite) status = fail(h, LES_ENONFINITE, "SOR residual is not finite");
    if (st) fill_stats(h, st, status);
    return status;
}

void member_set_dcur(les_s* h, int dcur) { h->dcur = dcur; }
int member_sweep(les_s* h, int in, int zero, cudaStream_t s) {
    if (h->sor.tile < 0) h->sor = SorCfg{6, 0};      // the ping-pong kernels only
    Geo<float> g = geo<float>(h);
    h->dcur = in;
    long long nl = 0;
    run_sweeps<float>(h, g, 1, zero, nl, s);
    h->launches += nl;
    return LES_OK;
}
int member_autotune(les_s* h, int sweeps) {
    double ms = 0.0;
    int rc = autotune_impl<float>(h, sweeps, &ms);
    if (h->sor.tile < 0) h->sor = SorCfg{6, 0};
    return rc;
}
bool member_net_on(const les_s* h) { return net_in_loop(h); }
int member_net_every(const les_s* h) { return h->net_every; }
void* member_rcur(les_s* h) { return net_in_loop(h) ? h->rcur : nullptr; }
int member_net_prepare(les_s* h) {
    if (!net_in_loop(h)) return LES_OK;
    return net_prepare(h->net, h->d, &h->net_gen);
}
long long member_net_generation(const les_s* h) { return net_in_loop(h) ? net_generation(h->net) : -1; }
int member_net_start(les_s* h, cudaStream_t s) {
    if (!(h->warm == LES_WARM_NET && h->net && h->prec == LES_FP32)) return LES_OK;
    if (!h->net_start && h->net_every > 0) return LES_OK;
    Geo<float> g = geo<float>(h);
    return net_correct<float>(h, g, s);
}
int member_net_loop(les_s* h, cudaStream_t s) {
    if (!net_in_loop(h)) return LES_OK;
    Geo<float> g = geo<float>(h);
    h->dcur = 0;
    return net_correct_loop<float>(h, g, s, true);
}
int member_parity(const les_s* h) { return h->cur; }
int member_begin(les_s* h, cudaStream_t s) {
    CK(cudaMemsetAsync(&h->sc->noconv_any, 0, sizeof(int), s));
    return LES_OK;
}
int* member_done_flag(les_s* h) { return &h->sc->done; }

}  // namespace les

