// Ensembles of uneven domains stepped together: every member is an ordinary
// FP32 domain handle (its own grid, buildings, inflow and state); the SOR
// solve of all members runs as batched launches over a flattened
// (member, tile) work list -- one persistent sweep launch per sweep (row
// tiles, or the members' TMA blocks with per-member tensor maps), one
// estimate launch and one refinement launch per batch for the whole ensemble
// -- each member gated by its own `done` flag, so members of different size
// stop at their own sweep counts.  Chunks of batches are captured in CUDA
// graphs; the last member to converge raises a mapped host flag.  Per member
// the arithmetic is the single-domain launch's, block for block, so a member
// of an ensemble evolves bit-identically to the same domain stepped alone with
// the same sweep tile.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <vector>

#include "../../include/les.h"
#include "les_internal.cuh"

using namespace les;

namespace {
constexpr int kEnsChunkBatches = 10;
// tile index of the per-member mode: every member sweeps with its own kernel
// and tile (TMA where its grid allows), one launch per member per sweep
constexpr int kPerMember = kNumEnsTiles;
// tile index of the batched TMA mode: one persistent launch per sweep walks
// the 28 x 8 x 8 TMA blocks of every member (tensor maps per member)
constexpr int kBatchedTma = kNumEnsTiles + 1;
}

struct les_ensemble_s {
    int n = 0;
    std::vector<les_handle> mem;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;                  // capture stream
    std::unique_ptr<EnsTab<float>> tab[2];      // per pressure-buffer parity
    int tile = 0;                                // ensemble row tile (0 .. kNumEnsTiles-1)
    int ctas = 0;                                // CTAs of the persistent sweep launch
    int check_every = 10;
    int cycle = 10;                              // sweeps per batch (check_every, or the network's interval)
    bool net = false;                            // members apply the learned correction in the loop
    std::vector<long long> net_gen;              // network workspace generation at capture
    int max_sweeps = 0;                          // largest member budget
    int cur = 0;                                 // parity of the members' pressure buffers
    int* ndone = nullptr;                        // device counter of members whose solve ended
    CUtensorMap* maps = nullptr;                 // 4 tensor maps per member (batched TMA mode), device
    bool persistent = false;                     // plain-SOR solves as one persistent launch per step
    unsigned* pbar = nullptr;                    // its grid-barrier state [2] and error flag
    int* perr = nullptr;
    int* all_done_host = nullptr;                // mapped pinned flag
    int* all_done_dev = nullptr;
    bool use_graph = true;
    bool graph_ok[2] = {false, false};
    cudaGraphExec_t chunk[2] = {nullptr, nullptr};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    long long launches = 0;
    char err[512] = {0};
};

namespace {

int efail(les_ensemble_s* e, int code, const char* fmt, ...) {
    if (e) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(e->err, sizeof e->err, fmt, ap);
        va_end(ap);
    }
    return code;
}

#define ECK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t err_ = (call);                                                                 \
        if (err_ != cudaSuccess) return efail(e, LES_ECUDA, "%s: %s", #call, cudaGetErrorString(err_)); \
    } while (0)

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// build both parity tables for the current tile
void fill_tables(les_ensemble_s* e) {
    for (int par = 0; par < 2; ++par) {
        EnsTab<float>& T = *e->tab[par];
        memset(&T, 0, sizeof T);
        T.n = e->n;
        T.tile = e->tile;
        T.ndone = e->ndone;
        T.all_done_host = e->all_done_dev;
        for (int i = 0; i < e->n; ++i) {
            les_handle h = e->mem[i];
            member_fill(h, T.m[i], e->tile >= kPerMember ? 0 : e->tile, par);
            T.sbeg[i + 1] = T.sbeg[i] + T.m[i].sgrid[0] * T.m[i].sgrid[1] * T.m[i].sgrid[2];
            T.ebeg[i + 1] = T.ebeg[i] + T.m[i].egrid[0] * T.m[i].egrid[1] * T.m[i].egrid[2];
            T.abeg[i + 1] = T.abeg[i] + T.m[i].agrid[0] * T.m[i].agrid[1] * T.m[i].agrid[2];
            T.rbeg[i + 1] = T.rbeg[i] + T.m[i].rblocks;
            const Dom& d = T.m[i].g.d;
            T.tbeg[i + 1] = T.tbeg[i] + ((d.nx + 27) / 28) * ((d.ny + kEnsTmaBy - 1) / kEnsTmaBy) *
                                            ((d.nz + kEnsTmaBz - 1) / kEnsTmaBz);
        }
    }
}

// the members' tensor maps of the batched TMA mode (device pointers of a
// member never change, so the maps are written once)
int fill_maps(les_ensemble_s* e) {
    std::vector<CUtensorMap> h(4 * (size_t)e->n);
    const EnsTab<float>& T = *e->tab[0];
    for (int i = 0; i < e->n; ++i) {
        const EnsMember<float>& M = T.m[i];
        if (!tma_encode_member(M.g.d, M.dl[0], M.dl[1], M.rr, M.g.flags, &h[4 * (size_t)i]))
            return efail(e, LES_ECUDA, "tensor maps of member %d could not be encoded", i);
    }
    ECK(cudaMemcpy(e->maps, h.data(), h.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    return LES_OK;
}

CondArgs eargs(const les_ensemble_s* e, int mode, int n, int gate) {
    CondArgs ca{};
    ca.mode = mode;
    ca.n = n;
    ca.gate = gate;
    ca.limit = e->max_sweeps;      // replaced per member inside the kernels
    ca.tol = 0.0;
    ca.done_host = nullptr;
    return ca;
}

// one chunk: kEnsChunkBatches x (cycle sweeps, estimate, gated refinement
// [, each member's network correction, done-gated])
int launch_chunk(les_ensemble_s* e, const EnsTab<float>& T, cudaStream_t s) {
    int dcur = 0;
    for (int b = 0; b < kEnsChunkBatches; ++b) {
        for (int q = 0; q < e->cycle; ++q) {
            if (e->tile == kPerMember) {
                for (les_handle h : e->mem) member_sweep(h, dcur, q == 0 ? 2 : 0, s);
                e->launches += e->n;
            } else if (e->tile == kBatchedTma) {
                e->launches += launch_sor_tma_ens(T, e->maps, dcur, q == 0 ? 2 : 0, e->ctas, s);
            } else {
                e->launches += launch_sor_ens(T, dcur, q == 0 ? 2 : 0, e->ctas, s);
            }
            dcur = 1 - dcur;
        }
        e->launches += launch_est_ens(T, dcur, eargs(e, RES_LOOP, e->cycle, 1), s);
        e->launches += launch_refine_ens(T, dcur, eargs(e, RES_LOOP, e->cycle, 1), s);
        if (e->net)
            for (les_handle h : e->mem) {
                int rc = member_net_loop(h, s);
                if (rc) return efail(e, rc, "member network correction: %s", les_last_error(h));
            }
    }
    ECK(cudaGetLastError());
    return LES_OK;
}

int build_chunk(les_ensemble_s* e, int par) {
    if (e->net)
        for (size_t i = 0; i < e->mem.size(); ++i) {
            // network workspaces are allocated before the capture
            int rc = member_net_prepare(e->mem[i]);
            if (rc) return efail(e, rc, "member network workspace: %s", les_last_error(e->mem[i]));
            e->net_gen[i] = member_net_generation(e->mem[i]);
        }
    ECK(cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeRelaxed));
    const long long l0 = e->launches;
    int rc = launch_chunk(e, *e->tab[par], e->cap);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(e->cap, &g);
    e->launches = l0;
    if (rc || ce != cudaSuccess) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        return efail(e, LES_ECUDA, "ensemble graph capture failed: %s", cudaGetErrorString(ce));
    }
    if (e->chunk[par]) cudaGraphExecDestroy(e->chunk[par]);
    e->chunk[par] = nullptr;
    ce = cudaGraphInstantiate(&e->chunk[par], g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        e->chunk[par] = nullptr;
        return efail(e, LES_ECUDA, "ensemble graph instantiate: %s", cudaGetErrorString(ce));
    }
    e->graph_ok[par] = true;
    return LES_OK;
}

void invalidate(les_ensemble_s* e) { e->graph_ok[0] = e->graph_ok[1] = false; }

int choose_ctas(les_ensemble_s* e, int per_sm) {
    if (e->tile == kPerMember) {
        e->ctas = 0;
        return LES_OK;
    }
    if (e->tile == kBatchedTma) {       // every resident CTA (the items are many small blocks)
        e->ctas = std::max(1, std::min(e->tab[0]->tbeg[e->n], sor_tma_ens_resident()));
        return LES_OK;
    }
    int occ = 0;
    // the sweep kernels are opted in to their shared memory at member creation
    const int smem = ens_rows_smem(e->tile);
    const int max_by_smem = std::max(1, (int)(227 * 1024 / std::max(smem, 1)));
    occ = std::min(per_sm, std::min(8, max_by_smem));
    const int total = e->tab[0]->sbeg[e->n];
    e->ctas = std::max(1, std::min(total, occ * sm_count()));
    return LES_OK;
}

void release(les_ensemble_s* e) {
    for (int c = 0; c < 2; ++c) {
        if (e->chunk[c]) cudaGraphExecDestroy(e->chunk[c]);
        if (e->ev[c]) cudaEventDestroy(e->ev[c]);
    }
    if (e->cap) cudaStreamDestroy(e->cap);
    if (e->ndone) cudaFree(e->ndone);
    if (e->maps) cudaFree(e->maps);
    if (e->pbar) cudaFree(e->pbar);
    if (e->perr) cudaFree(e->perr);
    if (e->all_done_host) cudaFreeHost(e->all_done_host);
    for (les_handle h : e->mem) les_destroy(h);
    e->mem.clear();
}

}  // namespace

extern "C" {

int les_ensemble_create(int32_t n, const les_grid_t* grids, const uint8_t* const* solid, const double* const* inflow,
                        void* stream, les_ensemble* out) {
    if (!out) return LES_EINVAL;
    *out = nullptr;
    if (n < 1 || n > kMaxMembers || !grids || !solid || !inflow) return LES_EINVAL;
    auto* e = new (std::nothrow) les_ensemble_s();
    if (!e) return LES_ENOMEM;
    e->n = n;
    e->stream = (cudaStream_t)stream;
    e->check_every = grids[0].check_every;
    for (int i = 0; i < n; ++i) {
        const les_grid_t& G = grids[i];
        int rc = LES_OK;
        if (G.precision != LES_FP32 || G.fixed_sweeps || G.check_every != e->check_every || G.check_every < 2 ||
            G.check_every % 2 || G.max_sweeps % G.check_every)
            rc = LES_EINVAL;
        les_handle h = nullptr;
        if (!rc) rc = les_create(&G, solid[i], inflow[i], stream, &h);
        if (rc) {
            snprintf(e->err, sizeof e->err,
                     "member %d: %s", i, rc == LES_EINVAL && !h
                                             ? "ensemble members need FP32, tolerance mode and a common even "
                                               "check_every dividing max_sweeps (or les_create rejected the grid)"
                                             : les_last_error(nullptr));
            release(e);
            delete e;
            return rc;
        }
        e->mem.push_back(h);
        e->max_sweeps = std::max(e->max_sweeps, G.max_sweeps);
    }
    int rc = LES_OK;
    for (int c = 0; c < 2 && !rc; ++c) {
        e->tab[c].reset(new (std::nothrow) EnsTab<float>());
        if (!e->tab[c]) rc = LES_ENOMEM;
    }
    if (!rc && cudaMalloc(&e->ndone, sizeof(int)) != cudaSuccess) rc = LES_ENOMEM;
    if (!rc && cudaMalloc(&e->maps, 4 * (size_t)n * sizeof(CUtensorMap)) != cudaSuccess) rc = LES_ENOMEM;
    if (!rc && cudaMalloc(&e->pbar, 2 * sizeof(unsigned)) != cudaSuccess) rc = LES_ENOMEM;
    if (!rc && cudaMalloc(&e->perr, sizeof(int)) != cudaSuccess) rc = LES_ENOMEM;
    if (!rc && cudaHostAlloc(&e->all_done_host, sizeof(int), cudaHostAllocMapped) != cudaSuccess) rc = LES_ENOMEM;
    if (!rc && cudaHostGetDevicePointer(&e->all_done_dev, e->all_done_host, 0) != cudaSuccess) rc = LES_ECUDA;
    if (!rc && cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking) != cudaSuccess) rc = LES_ECUDA;
    for (int c = 0; c < 2 && !rc; ++c)
        if (cudaEventCreateWithFlags(&e->ev[c], cudaEventDisableTiming) != cudaSuccess) rc = LES_ECUDA;
    if (rc) {
        release(e);
        delete e;
        return rc;
    }
    *e->all_done_host = 0;
    e->cycle = e->check_every;
    e->net_gen.assign(n, -1);
    e->tile = 0;
    fill_tables(e);
    choose_ctas(e, 4);
    if ((rc = fill_maps(e))) {
        release(e);
        delete e;
        return rc;
    }
    *out = e;
    return LES_OK;
}

void les_ensemble_destroy(les_ensemble e) {
    if (!e) return;
    cudaStreamSynchronize(e->stream);
    release(e);
    delete e;
}

const char* les_ensemble_last_error(les_ensemble e) { return e ? e->err : ""; }

int les_ensemble_size(les_ensemble e, int32_t* n) {
    if (!e || !n) return LES_EINVAL;
    *n = e->n;
    return LES_OK;
}

int les_ensemble_member(les_ensemble e, int32_t i, les_handle* out) {
    if (!e || !out) return LES_EINVAL;
    if (i < 0 || i >= e->n) return efail(e, LES_EINVAL, "member index %d out of range", i);
    *out = e->mem[i];
    return LES_OK;
}

int les_ensemble_set_graph(les_ensemble e, int32_t enable) {
    if (!e) return LES_EINVAL;
    e->use_graph = enable != 0;
    return LES_OK;
}

int les_ensemble_set_tile(les_ensemble e, int32_t tile, int32_t ctas_per_sm) {
    if (!e) return LES_EINVAL;
    if (tile < 0 || tile > kBatchedTma) return efail(e, LES_EINVAL, "tile must be 0..%d", kBatchedTma);
    if (ctas_per_sm < 1 || ctas_per_sm > 8) return efail(e, LES_EINVAL, "ctas_per_sm must be 1..8");
    e->tile = tile;
    fill_tables(e);
    choose_ctas(e, ctas_per_sm);
    invalidate(e);
    return LES_OK;
}

int les_ensemble_get_tile(les_ensemble e, int32_t* tile, int32_t* ctas) {
    if (!e || !tile || !ctas) return LES_EINVAL;
    *tile = e->tile;
    *ctas = e->ctas;
    return LES_OK;
}

int les_ensemble_step(les_ensemble e, int32_t nsteps, les_stats_t* stats) {
    if (!e) return LES_EINVAL;
    if (nsteps < 0) return efail(e, LES_EINVAL, "nsteps must be >= 0");
    cudaStream_t s = e->stream;
    for (les_handle h : e->mem)
        if (member_parity(h) != e->cur)
            return efail(e, LES_ESTATE, "a member was stepped on its own; step members only through the ensemble");
    for (les_handle h : e->mem) {
        int rc = member_begin(h, s);
        if (rc) return efail(e, rc, "member: %s", les_last_error(h));
    }
    const int per_chunk = kEnsChunkBatches * e->cycle;
    const int max_chunks = (e->max_sweeps + per_chunk - 1) / per_chunk + 1;
    for (int st = 0; st < nsteps; ++st) {
        const int par = e->cur;
        if (e->net)
            for (size_t i = 0; i < e->mem.size(); ++i)
                if (member_net_generation(e->mem[i]) != e->net_gen[i]) invalidate(e);
        if (e->use_graph && !e->graph_ok[par]) {
            if (build_chunk(e, par)) {
                e->use_graph = false;      // the same launches from the host from now on
                invalidate(e);
            }
        }
        ECK(cudaMemsetAsync(e->ndone, 0, sizeof(int), s));
        *(volatile int*)e->all_done_host = 0;
        for (les_handle h : e->mem) {
            const int rc = member_prefix(h, s);
            if (rc < 0) return efail(e, rc, "member prefix: %s", les_last_error(h));
            e->launches += rc;
        }
        const EnsTab<float>& T = *e->tab[par];
        e->launches += launch_refine_ens(T, 0, eargs(e, RES_INIT, 0, 0), s);
        if (e->net)
            for (les_handle h : e->mem) {
                int rc = member_net_start(h, s);
                if (rc) return efail(e, rc, "member network start: %s", les_last_error(h));
            }
        const bool persist = e->persistent && !e->net && e->tile == kBatchedTma;
        if (persist) {
            // the whole solve of every member in one cooperative launch
            ECK(cudaMemsetAsync(e->pbar, 0, 2 * sizeof(unsigned), s));
            ECK(cudaMemsetAsync(e->perr, 0, sizeof(int), s));
            const int batches = (e->max_sweeps + e->cycle - 1) / e->cycle + 1;
            const int rc = launch_ens_persist(T, e->maps, e->cycle, batches, eargs(e, RES_LOOP, e->cycle, 1), e->pbar,
                                              e->perr, s);
            if (rc < 0) return efail(e, LES_ECUDA, "the persistent ensemble solve could not be launched");
            e->launches += rc;
        }
        for (int c = 0; c < max_chunks && !persist; ++c) {
            if (e->use_graph) {
                ECK(cudaGraphLaunch(e->chunk[par], s));
                e->launches += kEnsChunkBatches * (e->cycle + 3 + (e->net ? 22 * e->n : 0));
            } else {
                int rc = launch_chunk(e, T, s);
                if (rc) return rc;
            }
            ECK(cudaEventRecord(e->ev[c & 1], s));
            if (c >= 1) {
                ECK(cudaEventSynchronize(e->ev[(c - 1) & 1]));
                if (*(volatile int*)e->all_done_host) break;
            }
        }
        for (les_handle h : e->mem) {
            member_set_dcur(h, 0);
            int rc = member_finish(h, s);
            if (rc) return efail(e, rc, "member projection: %s", les_last_error(h));
        }
        e->launches += e->n;
        e->cur = 1 - e->cur;
    }
    ECK(cudaStreamSynchronize(s));
    if (e->persistent) {
        int perr = 0;
        ECK(cudaMemcpy(&perr, e->perr, sizeof(int), cudaMemcpyDeviceToHost));
        if (perr) return efail(e, LES_ETIMEOUT, "a bounded wait of the persistent ensemble solve timed out");
    }
    int worst = LES_OK;
    for (int i = 0; i < e->n; ++i) {
        int rc = member_stats(e->mem[i], stats ? &stats[i] : nullptr);
        if (rc < 0) return efail(e, rc, "member %d: %s", i, les_last_error(e->mem[i]));
        if (rc == LES_ENOCONV) worst = LES_ENOCONV;
    }
    return worst;
}

int les_ensemble_autotune(les_ensemble e, int32_t sweeps, double* best_ms_per_sweep) {
    if (!e) return LES_EINVAL;
    if (sweeps < 1) return efail(e, LES_EINVAL, "sweeps must be >= 1");
    cudaStream_t s = e->stream;
    cudaEvent_t a, b;
    ECK(cudaEventCreate(&a));
    ECK(cudaEventCreate(&b));
    // the timed sweeps touch only the members' correction buffers; their
    // `done` flags are cleared for the timing and put back afterwards
    std::vector<int> keep(e->n, 0);
    for (int i = 0; i < e->n; ++i)
        ECK(cudaMemcpyAsync(&keep[i], member_done_flag(e->mem[i]), sizeof(int), cudaMemcpyDeviceToHost, s));
    ECK(cudaStreamSynchronize(s));
    for (int i = 0; i < e->n; ++i) ECK(cudaMemsetAsync(member_done_flag(e->mem[i]), 0, sizeof(int), s));
    const int tile0 = e->tile, ctas0 = e->ctas;
    int best_tile = tile0, best_per_sm = 4;
    double best = 1e300;
    const int per_sm_opts[] = {2, 4, 6, 8};
    for (int t = 0; t < kNumEnsTiles; ++t)
        for (int per_sm : per_sm_opts) {
            e->tile = t;
            fill_tables(e);
            choose_ctas(e, per_sm);
            const EnsTab<float>& T = *e->tab[e->cur];
            launch_sor_ens(T, 0, 0, e->ctas, s);
            launch_sor_ens(T, 1, 0, e->ctas, s);
            ECK(cudaEventRecord(a, s));
            for (int q = 0; q < sweeps; ++q) launch_sor_ens(T, q & 1, 0, e->ctas, s);
            ECK(cudaEventRecord(b, s));
            ECK(cudaEventSynchronize(b));
            ECK(cudaGetLastError());
            float ms = 0.f;
            ECK(cudaEventElapsedTime(&ms, a, b));
            if (ms / sweeps < best) {
                best = ms / sweeps;
                best_tile = t;
                best_per_sm = per_sm;
            }
        }
    {
        // the per-member mode: each member first picks its own kernel and tile
        for (les_handle h : e->mem) {
            int rc = member_autotune(h, std::max(2, sweeps / 2));
            if (rc) return efail(e, rc, "member autotune: %s", les_last_error(h));
        }
        for (int i = 0; i < e->n; ++i) ECK(cudaMemsetAsync(member_done_flag(e->mem[i]), 0, sizeof(int), s));
        for (les_handle h : e->mem) {
            member_sweep(h, 0, 0, s);
            member_sweep(h, 1, 0, s);
        }
        ECK(cudaEventRecord(a, s));
        for (int q = 0; q < sweeps; ++q)
            for (les_handle h : e->mem) member_sweep(h, q & 1, 0, s);
        ECK(cudaEventRecord(b, s));
        ECK(cudaEventSynchronize(b));
        ECK(cudaGetLastError());
        float ms = 0.f;
        ECK(cudaEventElapsedTime(&ms, a, b));
        for (les_handle h : e->mem) member_set_dcur(h, 0);
        if (ms / sweeps < best) {
            best = ms / sweeps;
            best_tile = kPerMember;
        }
    }
    {
        // the batched TMA mode: one persistent launch per sweep over every member's blocks
        e->tile = kBatchedTma;
        fill_tables(e);
        choose_ctas(e, 4);
        const EnsTab<float>& T = *e->tab[e->cur];
        launch_sor_tma_ens(T, e->maps, 0, 0, e->ctas, s);
        launch_sor_tma_ens(T, e->maps, 1, 0, e->ctas, s);
        ECK(cudaEventRecord(a, s));
        for (int q = 0; q < sweeps; ++q) launch_sor_tma_ens(T, e->maps, q & 1, 0, e->ctas, s);
        ECK(cudaEventRecord(b, s));
        ECK(cudaEventSynchronize(b));
        ECK(cudaGetLastError());
        float ms = 0.f;
        ECK(cudaEventElapsedTime(&ms, a, b));
        if (ms / sweeps < best) {
            best = ms / sweeps;
            best_tile = kBatchedTma;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    for (int i = 0; i < e->n; ++i)
        ECK(cudaMemcpyAsync(member_done_flag(e->mem[i]), &keep[i], sizeof(int), cudaMemcpyHostToDevice, s));
    ECK(cudaStreamSynchronize(s));
    (void)ctas0;
    e->tile = best_tile;
    fill_tables(e);
    choose_ctas(e, best_per_sm);
    invalidate(e);
    if (best_ms_per_sweep) *best_ms_per_sweep = best;
    return LES_OK;
}

int les_ensemble_set_warmstart(les_ensemble e, les_net net, int32_t every_sweeps) {
    if (!e) return LES_EINVAL;
    if (net && (every_sweeps < 2 || every_sweeps % 2))
        return efail(e, LES_EINVAL, "every_sweeps must be even and >= 2");
    for (les_handle h : e->mem)
        if (net && member_max_sweeps(h) % every_sweeps)
            return efail(e, LES_EINVAL, "every_sweeps must divide each member's max_sweeps");
    for (les_handle h : e->mem) {
        int rc = net ? les_set_warmstart(h, LES_WARM_NET, net) : les_set_warmstart(h, LES_WARM_PREV, nullptr);
        if (!rc) rc = les_set_net_schedule(h, net ? every_sweeps : 0);
        if (rc) return efail(e, rc, "member: %s", les_last_error(h));
    }
    e->net = net != nullptr;
    e->cycle = net ? every_sweeps : e->check_every;
    e->net_gen.assign(e->mem.size(), -1);
    fill_tables(e);
    invalidate(e);
    return LES_OK;
}

int les_ensemble_set_persistent(les_ensemble e, int32_t enable) {
    if (!e) return LES_EINVAL;
    if (enable && ens_persist_grid() <= 0)
        return efail(e, LES_EINVAL, "this device cannot run the cooperative persistent solve");
    e->persistent = enable != 0;
    if (e->persistent && e->tile != kBatchedTma) {
        e->tile = kBatchedTma;
        fill_tables(e);
        choose_ctas(e, 4);
        invalidate(e);
    }
    return LES_OK;
}

int les_ensemble_launches(les_ensemble e, int64_t* launches) {
    if (!e || !launches) return LES_EINVAL;
    *launches = e->launches;
    return LES_OK;
}

}  // extern "C"
