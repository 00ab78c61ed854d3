// The learned SOR warm start: a 4-level 3-D U-Net (16, 32, 64, 128
// channels) on BF16 activations with FP32 accumulation (kernels in
// les_nn_kernels.cu), trained on the GPU with its own forward / backward
// kernels and Adam.  The paper has no learned component; this implements the
// warm start described by the entry points in include/les.h.
//
// Network (bias-free, so it is positively homogeneous: scaling the input
// scales the output):
//   e0 = relu(c0(x))            16 @ level 0   x: residual / rms, fluid mask
//   e1 = relu(c1(pool e0))      32 @ level 1
//   e2 = relu(c2(pool e1))      64 @ level 2
//   e3 = relu(c3(pool e2))     128 @ level 3
//   d2 = relu(c4(up e3)) + e2   64 @ level 2
//   d1 = relu(c5(up d2)) + e1   32 @ level 1
//   d0 = relu(c6(up d1)) + e0   16 @ level 0
//   y  = mask * (w_head . d0)    1 @ level 0  (FP32)
// c* are 3x3x3 convolutions with zero padding; pool = 2x2x2 mean, up =
// nearest.  Training minimises mean_fluid (y - t / rms(t))^2: the net
// predicts the direction of the pressure correction, and the solver scales
// it by an FP64 line search.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/les.h"
#include "les_nn.cuh"

using namespace les;

namespace {

constexpr int kConvs = 7;
const int kCin[kConvs] = {16, 16, 32, 64, 128, 64, 32};
const int kCout[kConvs] = {16, 32, 64, 128, 64, 32, 16};
constexpr int kHeadC = 16;

struct Level {
    int X, Y, Z;
    size_t v() const { return (size_t)X * Y * Z; }
};

// splitmix64 + Box-Muller, counter based (same construction as the inflow noise)
uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double normal_at(uint64_t seed, uint64_t c) {
    auto u = [&](uint64_t k) {
        return ((double)(mix64(seed + (k + 1) * 0x9E3779B97F4A7C15ull) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    return std::sqrt(-2.0 * std::log(u(2 * c))) * std::cos(6.283185307179586 * u(2 * c + 1));
}

// per-sample RMS over the mask, rms = sqrt(sum mask*a^2 / sum mask), in a
// fixed summation order (the result must not depend on scheduling): each
// block writes its two partial sums to part[2*block], k_rms_final adds the
// partials in block order into out[0] (rms) and out[1] (sum of the mask)
constexpr int kRmsBlocks = 256;
// input-channel split workspace: up to 2 CTAs per SM x 256 threads x 8 floats
constexpr size_t kSplitFloats = (size_t)2 * 160 * 256 * 8;
constexpr size_t kSplitCounters = 4096;
__global__ void __launch_bounds__(256) k_rms(const float* a, const float* mask, size_t n, double* part,
                                             const int* gate) {
    if (gate && *(volatile const int*)gate) return;
    __shared__ double sh[2][8];
    double s = 0.0, m = 0.0;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const double v = a[q], w = mask[q];
        s += w * v * v;
        m += w;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        m += __shfl_down_sync(0xffffffffu, m, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][warp] = s;
        sh[1][warp] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ts = 0.0, tm = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            ts += sh[0][w];
            tm += sh[1][w];
        }
        part[2 * blockIdx.x] = ts;
        part[2 * blockIdx.x + 1] = tm;
    }
}
// one block of kRmsBlocks threads: thread b takes partial b, then a fixed
// shared-memory tree (deterministic)
__global__ void __launch_bounds__(kRmsBlocks) k_rms_final(const double* part, int nblocks, double* out,
                                                          const int* gate) {
    if (gate && *(volatile const int*)gate) return;
    __shared__ double ss[kRmsBlocks], sm[kRmsBlocks];
    const int t = threadIdx.x;
    ss[t] = t < nblocks ? part[2 * t] : 0.0;
    sm[t] = t < nblocks ? part[2 * t + 1] : 0.0;
    __syncthreads();
    for (int o = kRmsBlocks / 2; o > 0; o >>= 1) {
        if (t < o) {
            ss[t] += ss[t + o];
            sm[t] += sm[t + o];
        }
        __syncthreads();
    }
    if (t == 0) {
        out[0] = sm[0] > 0.0 ? sqrt(ss[0] / sm[0]) : 0.0;
        out[1] = sm[0];
    }
}
// dense input: channel 0 = r / scale, channel 1 = mask
__global__ void k_pack_dense(const float* r, const float* mask, const double* scale, __nv_bfloat16* xin, size_t n,
                             const int* gate) {
    pdl_wait();
    if (gate && *(volatile const int*)gate) return;
    const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const float s = (float)(scale[0] > 0.0 ? 1.0 / scale[0] : 0.0);
    __nv_bfloat16* o = xin + v * 16;
    o[0] = __float2bfloat16(mask[v] * r[v] * s);
    o[1] = __float2bfloat16(mask[v]);
    for (int c = 2; c < 16; ++c) o[c] = __float2bfloat16(0.f);
}
__global__ void k_scale(const float* a, const double* scale, float* b, size_t n) {
    const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    b[v] = (float)(scale[0] > 0.0 ? a[v] / scale[0] : 0.0);
}

}  // namespace

struct les_net_s {
    cudaStream_t stream = nullptr;
    // FP32 master parameters (flat: conv0..conv6 [27][Cout][Cin], head [16]) and Adam state
    size_t off[kConvs + 1];
    size_t nparam = 0;
    float *w32 = nullptr, *g32 = nullptr, *m32 = nullptr, *v32 = nullptr;
    __nv_bfloat16* wb[kConvs] = {};     // BF16 copies
    __nv_bfloat16* wt[kConvs] = {};     // flipped copies for the input gradient
    long long adam_t = 0;
    std::vector<void*> owned;
    // activation workspace, sized per level for the largest volumes seen so far
    size_t cap_v0 = 0;
    size_t cap[4] = {0, 0, 0, 0};
    std::vector<void*> ws;
    __nv_bfloat16 *xin = nullptr, *e[4] = {}, *p[3] = {}, *u[3] = {}, *r[3] = {}, *dd[3] = {};
    __nv_bfloat16 *ga = nullptr, *gb = nullptr, *gd0 = nullptr, *gd1 = nullptr, *gd2 = nullptr, *ge3 = nullptr,
                  *gpb = nullptr;
    float *y = nullptr, *gy = nullptr, *mask = nullptr, *tn = nullptr;
    int stride = 1;                     // the network runs on the grid coarsened stride times per axis
    int engine = nn::kEngineTcgen05;    // forward convolutions: tcgen05 (default) or warp-level mma.sync
    int* tc_timeout = nullptr;          // device flag: a bounded wait of a tcgen05 convolution gave up
    float *rc = nullptr, *mc = nullptr, *tc = nullptr;     // pooled sample (coarse level 0)
    double* dscal = nullptr;            // [0,1] rms / mask sum of r, [2,3] of t, [62] loss, [64..) partials
    long long ws_gen = 0;               // bumped whenever the workspace is reallocated
    // persistent inference: per-CTA sums, grid barrier state
    double* cta = nullptr;              // [4 * kMaxInferGrid]
    unsigned* bar = nullptr;            // [2]: count, generation
    double* pp_part = nullptr;          // [2 * kPoolRmsMax] per-block partials of the pooling + RMS kernel
    unsigned* pp_count = nullptr;       // its completion counter (zero between launches)
    nn::ConvSplit split = {};           // input-channel split workspace of the inference convolutions
    int last_launches = 0;              // kernels of the last inference
    char err[256] = {0};
};

namespace {

constexpr int kMaxInferGrid = 1024;

int nfail(les_net_s* n, int code, const char* msg, cudaError_t e = cudaSuccess) {
    if (n)
        snprintf(n->err, sizeof n->err, "%s%s%s", msg, e != cudaSuccess ? ": " : "",
                 e != cudaSuccess ? cudaGetErrorString(e) : "");
    return code;
}
#define NCK(call)                                                     \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return nfail(n, LES_ECUDA, #call, e_); \
    } while (0)

Level level(const Level& l0, int l) {
    Level o = l0;
    for (int i = 0; i < l; ++i) o = Level{(o.X + 1) / 2, (o.Y + 1) / 2, (o.Z + 1) / 2};
    return o;
}

// the network's level 0 for a fine grid
Level coarse(const les_net_s* n, const Level& f) {
    const int s = n->stride;
    return Level{(f.X + s - 1) / s, (f.Y + s - 1) / s, (f.Z + s - 1) / s};
}

void free_ws(les_net_s* n) {
    for (void* q : n->ws) cudaFree(q);
    n->ws.clear();
    n->cap_v0 = 0;
    for (size_t& c : n->cap) c = 0;
}

// every buffer is sized from each level's volume (grown by 25% so nearby
// shapes reuse the workspace); a shape that exceeds any level reallocates
int ensure_ws(les_net_s* n, const Level& L0) {
    Level Lb[4];
    for (int l = 0; l < 4; ++l) Lb[l] = level(L0, l);
    bool fits = n->cap_v0 > 0;
    for (int l = 0; l < 4 && fits; ++l) fits = Lb[l].v() <= n->cap[l];
    if (fits) return LES_OK;
    NCK(cudaStreamSynchronize(n->stream));
    size_t want[4];
    for (int l = 0; l < 4; ++l) {
        const size_t v = Lb[l].v() + Lb[l].v() / 4 + 64;
        want[l] = v > n->cap[l] ? v : n->cap[l];
    }
    free_ws(n);
    auto vol = [&](int l) { return want[l]; };
    auto get = [&](size_t elems, size_t es, void** q) -> int {
        cudaError_t e = cudaMalloc(q, elems * es);
        if (e != cudaSuccess) return nfail(n, LES_ENOMEM, "network workspace", e);
        n->ws.push_back(*q);
        return LES_OK;
    };
    const size_t B = sizeof(__nv_bfloat16);
    int rc;
    const int ce[4] = {16, 32, 64, 128};
    if ((rc = get(vol(0) * 16, B, (void**)&n->xin))) return rc;
    for (int l = 0; l < 4; ++l)
        if ((rc = get(vol(l) * ce[l], B, (void**)&n->e[l]))) return rc;
    for (int l = 0; l < 3; ++l) {
        if ((rc = get(vol(l + 1) * ce[l], B, (void**)&n->p[l]))) return rc;      // pool(e_l), level l+1
        if ((rc = get(vol(l) * ce[l + 1], B, (void**)&n->u[l]))) return rc;      // up(d_{l+1} | e_3), level l
        if ((rc = get(vol(l) * ce[l], B, (void**)&n->r[l]))) return rc;          // relu(conv), level l
        if ((rc = get(vol(l) * ce[l], B, (void**)&n->dd[l]))) return rc;         // d_l
    }
    size_t gmax = 0;
    for (int l = 0; l < 4; ++l) {
        const size_t c = vol(l) * (size_t)(l < 3 ? ce[l + 1] : ce[3]);
        gmax = c > gmax ? c : gmax;
    }
    if ((rc = get(gmax, B, (void**)&n->ga))) return rc;
    if ((rc = get(gmax, B, (void**)&n->gb))) return rc;
    if ((rc = get(vol(0) * 16, B, (void**)&n->gd0))) return rc;
    if ((rc = get(vol(1) * 32, B, (void**)&n->gd1))) return rc;
    if ((rc = get(vol(2) * 64, B, (void**)&n->gd2))) return rc;
    if ((rc = get(vol(3) * 128, B, (void**)&n->ge3))) return rc;
    // pooled-branch gradient: level l (l = 0..2) with ce[l] channels
    size_t pmax = 0;
    for (int l = 0; l < 3; ++l) pmax = vol(l) * ce[l] > pmax ? vol(l) * ce[l] : pmax;
    if ((rc = get(pmax, B, (void**)&n->gpb))) return rc;
    if ((rc = get(vol(0), sizeof(float), (void**)&n->y))) return rc;
    if ((rc = get(vol(0), sizeof(float), (void**)&n->gy))) return rc;
    if ((rc = get(vol(0), sizeof(float), (void**)&n->mask))) return rc;
    if ((rc = get(vol(0), sizeof(float), (void**)&n->tn))) return rc;
    if ((rc = get(vol(0), sizeof(float), (void**)&n->rc))) return rc;
    if ((rc = get(vol(0), sizeof(float), (void**)&n->mc))) return rc;
    if ((rc = get(vol(0), sizeof(float), (void**)&n->tc))) return rc;
    if ((rc = get(64 + 4 * kRmsBlocks, sizeof(double), (void**)&n->dscal))) return rc;
    for (int l = 0; l < 4; ++l) n->cap[l] = want[l];
    n->cap_v0 = want[0];
    n->ws_gen += 1;
    return LES_OK;
}

// inference forward: pooling and upsampling folded into the convolutions'
// input staging (bit-identical to forward(), which keeps the pooled and
// upsampled tensors for the backward pass); every kernel returns at once
// while *gate != 0 (gate may be null)
void forward_fused(les_net_s* n, const Level& L0, const int* gate) {
    cudaStream_t s = n->stream;
    const Level L1 = level(L0, 1), L2 = level(L0, 2), L3 = level(L0, 3);
    const nn::ConvSplit* sp = &n->split;
    nn::conv3_fwd(n->xin, n->wb[0], n->e[0], nullptr, nullptr, L0.X, L0.Y, L0.Z, 16, 16, 1, s, gate, sp);
    nn::conv3_fwd_pool(n->e[0], n->wb[1], n->e[1], L0.X, L0.Y, L0.Z, 16, 32, 1, s, gate, sp);
    nn::conv3_fwd_pool(n->e[1], n->wb[2], n->e[2], L1.X, L1.Y, L1.Z, 32, 64, 1, s, gate, sp);
    nn::conv3_fwd_pool(n->e[2], n->wb[3], n->e[3], L2.X, L2.Y, L2.Z, 64, 128, 1, s, gate, sp);
    nn::conv3_fwd_up(n->e[3], n->wb[4], n->r[2], n->e[2], n->dd[2], L2.X, L2.Y, L2.Z, 128, 64, 1, s, gate, sp);
    nn::conv3_fwd_up(n->dd[2], n->wb[5], n->r[1], n->e[1], n->dd[1], L1.X, L1.Y, L1.Z, 64, 32, 1, s, gate, sp);
    nn::conv3_fwd_up(n->dd[1], n->wb[6], n->r[0], n->e[0], n->dd[0], L0.X, L0.Y, L0.Z, 32, 16, 1, s, gate, sp);
    nn::head(n->dd[0], n->w32 + n->off[kConvs], n->mask, n->y, L0.v(), kHeadC, s, gate);
}

// the same on the tcgen05 engine with the packing folded into the first
// convolution's staging (input from the pooled residual n->rc, the pooled
// mask n->mask and the RMS n->dscal[0]) and the head into the last one's
// epilogue; the values are those of forward_fused after k_pack_dense
void forward_tc_folded(les_net_s* n, const Level& L0, const int* gate) {
    cudaStream_t s = n->stream;
    const Level L1 = level(L0, 1), L2 = level(L0, 2);
    const nn::ConvSplit* sp = &n->split;
    nn::conv3_tc_fwd_packed(n->rc, n->mask, n->dscal, n->wb[0], n->e[0], L0.X, L0.Y, L0.Z, 16, 1, s, gate, sp);
    nn::conv3_fwd_pool(n->e[0], n->wb[1], n->e[1], L0.X, L0.Y, L0.Z, 16, 32, 1, s, gate, sp);
    nn::conv3_fwd_pool(n->e[1], n->wb[2], n->e[2], L1.X, L1.Y, L1.Z, 32, 64, 1, s, gate, sp);
    nn::conv3_fwd_pool(n->e[2], n->wb[3], n->e[3], L2.X, L2.Y, L2.Z, 64, 128, 1, s, gate, sp);
    nn::conv3_fwd_up(n->e[3], n->wb[4], n->r[2], n->e[2], n->dd[2], L2.X, L2.Y, L2.Z, 128, 64, 1, s, gate, sp);
    nn::conv3_fwd_up(n->dd[2], n->wb[5], n->r[1], n->e[1], n->dd[1], L1.X, L1.Y, L1.Z, 64, 32, 1, s, gate, sp);
    nn::conv3_tc_fwd_up_head(n->dd[1], n->wb[6], n->e[0], L0.X, L0.Y, L0.Z, 32, 1, n->w32 + n->off[kConvs], n->mask,
                             n->y, s, gate, sp);
}

// forward on the packed input n->xin with mask n->mask; output n->y
// (every kernel returns at once while *gate != 0; gate may be null)
void forward(les_net_s* n, const Level& L0, const int* gate = nullptr) {
    cudaStream_t s = n->stream;
    const Level L1 = level(L0, 1), L2 = level(L0, 2), L3 = level(L0, 3);
    nn::conv3_fwd(n->xin, n->wb[0], n->e[0], nullptr, nullptr, L0.X, L0.Y, L0.Z, 16, 16, 1, s, gate);
    nn::pool(n->e[0], n->p[0], L0.X, L0.Y, L0.Z, 16, s, gate);
    nn::conv3_fwd(n->p[0], n->wb[1], n->e[1], nullptr, nullptr, L1.X, L1.Y, L1.Z, 16, 32, 1, s, gate);
    nn::pool(n->e[1], n->p[1], L1.X, L1.Y, L1.Z, 32, s, gate);
    nn::conv3_fwd(n->p[1], n->wb[2], n->e[2], nullptr, nullptr, L2.X, L2.Y, L2.Z, 32, 64, 1, s, gate);
    nn::pool(n->e[2], n->p[2], L2.X, L2.Y, L2.Z, 64, s, gate);
    nn::conv3_fwd(n->p[2], n->wb[3], n->e[3], nullptr, nullptr, L3.X, L3.Y, L3.Z, 64, 128, 1, s, gate);
    nn::up(n->e[3], n->u[2], L2.X, L2.Y, L2.Z, 128, s, gate);
    nn::conv3_fwd(n->u[2], n->wb[4], n->r[2], n->e[2], n->dd[2], L2.X, L2.Y, L2.Z, 128, 64, 1, s, gate);
    nn::up(n->dd[2], n->u[1], L1.X, L1.Y, L1.Z, 64, s, gate);
    nn::conv3_fwd(n->u[1], n->wb[5], n->r[1], n->e[1], n->dd[1], L1.X, L1.Y, L1.Z, 64, 32, 1, s, gate);
    nn::up(n->dd[1], n->u[0], L0.X, L0.Y, L0.Z, 32, s, gate);
    nn::conv3_fwd(n->u[0], n->wb[6], n->r[0], n->e[0], n->dd[0], L0.X, L0.Y, L0.Z, 32, 16, 1, s, gate);
    nn::head(n->dd[0], n->w32 + n->off[kConvs], n->mask, n->y, L0.v(), kHeadC, s, gate);
}

// backward from n->gy; accumulates the parameter gradients into n->g32
void backward(les_net_s* n, const Level& L0) {
    cudaStream_t s = n->stream;
    const Level L1 = level(L0, 1), L2 = level(L0, 2), L3 = level(L0, 3);
    float* G = n->g32;
    auto gw = [&](int c) { return G + n->off[c]; };
    nn::head_bwd(n->dd[0], n->w32 + n->off[kConvs], n->mask, n->gy, n->gd0, G + n->off[kConvs], L0.v(), kHeadC, s);
    // d0 = relu(c6(u0)) + e0
    nn::relu_bwd(n->r[0], n->gd0, nullptr, n->ga, L0.v() * 16, s);
    nn::conv3_wgrad(n->u[0], n->ga, gw(6), L0.X, L0.Y, L0.Z, 32, 16, s);
    nn::conv3_fwd(n->ga, n->wt[6], n->gb, nullptr, nullptr, L0.X, L0.Y, L0.Z, 16, 32, 0, s);
    nn::up_bwd(n->gb, n->gd1, L0.X, L0.Y, L0.Z, 32, s);
    // d1 = relu(c5(u1)) + e1
    nn::relu_bwd(n->r[1], n->gd1, nullptr, n->ga, L1.v() * 32, s);
    nn::conv3_wgrad(n->u[1], n->ga, gw(5), L1.X, L1.Y, L1.Z, 64, 32, s);
    nn::conv3_fwd(n->ga, n->wt[5], n->gb, nullptr, nullptr, L1.X, L1.Y, L1.Z, 32, 64, 0, s);
    nn::up_bwd(n->gb, n->gd2, L1.X, L1.Y, L1.Z, 64, s);
    // d2 = relu(c4(u2)) + e2
    nn::relu_bwd(n->r[2], n->gd2, nullptr, n->ga, L2.v() * 64, s);
    nn::conv3_wgrad(n->u[2], n->ga, gw(4), L2.X, L2.Y, L2.Z, 128, 64, s);
    nn::conv3_fwd(n->ga, n->wt[4], n->gb, nullptr, nullptr, L2.X, L2.Y, L2.Z, 64, 128, 0, s);
    nn::up_bwd(n->gb, n->ge3, L2.X, L2.Y, L2.Z, 128, s);
    // e3 = relu(c3(p2))
    nn::relu_bwd(n->e[3], n->ge3, nullptr, n->ga, L3.v() * 128, s);
    nn::conv3_wgrad(n->p[2], n->ga, gw(3), L3.X, L3.Y, L3.Z, 64, 128, s);
    nn::conv3_fwd(n->ga, n->wt[3], n->gb, nullptr, nullptr, L3.X, L3.Y, L3.Z, 128, 64, 0, s);
    nn::pool_bwd(n->gb, n->gpb, L2.X, L2.Y, L2.Z, 64, s);
    // e2 = relu(c2(p1)); dL/de2 = skip part + pooled part
    nn::relu_bwd(n->e[2], n->gd2, n->gpb, n->ga, L2.v() * 64, s);
    nn::conv3_wgrad(n->p[1], n->ga, gw(2), L2.X, L2.Y, L2.Z, 32, 64, s);
    nn::conv3_fwd(n->ga, n->wt[2], n->gb, nullptr, nullptr, L2.X, L2.Y, L2.Z, 64, 32, 0, s);
    nn::pool_bwd(n->gb, n->gpb, L1.X, L1.Y, L1.Z, 32, s);
    // e1 = relu(c1(p0))
    nn::relu_bwd(n->e[1], n->gd1, n->gpb, n->ga, L1.v() * 32, s);
    nn::conv3_wgrad(n->p[0], n->ga, gw(1), L1.X, L1.Y, L1.Z, 16, 32, s);
    nn::conv3_fwd(n->ga, n->wt[1], n->gb, nullptr, nullptr, L1.X, L1.Y, L1.Z, 32, 16, 0, s);
    nn::pool_bwd(n->gb, n->gpb, L0.X, L0.Y, L0.Z, 16, s);
    // e0 = relu(c0(xin))
    nn::relu_bwd(n->e[0], n->gd0, n->gpb, n->ga, L0.v() * 16, s);
    nn::conv3_wgrad(n->xin, n->ga, gw(0), L0.X, L0.Y, L0.Z, 16, 16, s);
}

void refresh_copies(les_net_s* n) {
    for (int c = 0; c < kConvs; ++c) {
        const size_t cnt = (size_t)27 * kCin[c] * kCout[c];
        nn::to_bf16(n->w32 + n->off[c], n->wb[c], cnt, n->stream);
        nn::wflip(n->wb[c], n->wt[c], kCin[c], kCout[c], n->stream);
    }
}

// pack a dense coarse sample (r, mask, optional target t) into the network
// input and normalise the target; nmask receives sum(mask) when asked
int pack_sample(les_net_s* n, const Level& L0, const float* r, const float* mask, const float* t, double* nmask,
                const int* gate = nullptr) {
    const size_t v = L0.v();
    cudaStream_t s = n->stream;
    const int blocks = (int)((v + 255) / 256 < (size_t)kRmsBlocks ? (v + 255) / 256 : kRmsBlocks);
    double* part = n->dscal + 64;
    k_rms<<<blocks, 256, 0, s>>>(r, mask, v, part, gate);
    k_rms_final<<<1, kRmsBlocks, 0, s>>>(part, blocks, n->dscal, gate);
    if (t) {
        k_rms<<<blocks, 256, 0, s>>>(t, mask, v, part + 2 * kRmsBlocks, gate);
        k_rms_final<<<1, kRmsBlocks, 0, s>>>(part + 2 * kRmsBlocks, blocks, n->dscal + 2, gate);
    }
    if (mask != n->mask) NCK(cudaMemcpyAsync(n->mask, mask, v * sizeof(float), cudaMemcpyDeviceToDevice, s));
    k_pack_dense<<<(unsigned)((v + 255) / 256), 256, 0, s>>>(r, n->mask, n->dscal, n->xin, v, gate);
    if (t) k_scale<<<(unsigned)((v + 255) / 256), 256, 0, s>>>(t, n->dscal + 2, n->tn, v);
    NCK(cudaGetLastError());
    if (nmask) {
        double host[2];
        NCK(cudaMemcpyAsync(host, n->dscal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        NCK(cudaStreamSynchronize(s));
        *nmask = host[1];
    }
    return LES_OK;
}

// sample b of a dense fine batch: pooled to the network's level 0 when the
// stride is above 1, then packed
int prepare_sample(les_net_s* n, const Level& Lf, const float* r, const float* mask, const float* t, size_t b,
                   double* nmask) {
    const size_t vf = Lf.v();
    const float *pr = r + b * vf, *pm = mask + b * vf, *pt = t ? t + b * vf : nullptr;
    if (n->stride > 1) {
        const int st = n->stride;
        nn::pool_dense_s(pr, n->rc, Lf.X, Lf.Y, Lf.Z, st, n->stream);
        nn::pool_dense_s(pm, n->mc, Lf.X, Lf.Y, Lf.Z, st, n->stream);
        if (pt) nn::pool_dense_s(pt, n->tc, Lf.X, Lf.Y, Lf.Z, st, n->stream);
        pr = n->rc;
        pm = n->mc;
        pt = pt ? n->tc : nullptr;
    }
    return pack_sample(n, coarse(n, Lf), pr, pm, pt, nmask);
}

// forward + loss + backward over a batch, gradients accumulated in g32
int batch_grad(les_net_s* n, const Level& Lf, const float* r, const float* mask, const float* t, int B, double* loss) {
    const Level L0 = coarse(n, Lf);
    int rc = ensure_ws(n, L0);
    if (rc) return rc;
    cudaStream_t s = n->stream;
    NCK(cudaMemsetAsync(n->g32, 0, n->nparam * sizeof(float), s));
    double* dl = n->dscal + 62;
    NCK(cudaMemsetAsync(dl, 0, sizeof(double), s));
    for (int b = 0; b < B; ++b) {
        double nm = 0.0;
        if ((rc = prepare_sample(n, Lf, r, mask, t, b, &nm))) return rc;
        forward(n, L0);
        const double inv = nm > 0.0 ? 1.0 / (nm * B) : 0.0;
        nn::mse(n->y, n->tn, n->mask, n->gy, dl, L0.v(), inv, s);
        backward(n, L0);
        NCK(cudaGetLastError());
    }
    NCK(cudaMemcpyAsync(loss, dl, sizeof(double), cudaMemcpyDeviceToHost, s));
    NCK(cudaStreamSynchronize(s));
    return LES_OK;
}

}  // namespace

// ===========================================================================
// solver-side inference (les_api.cu): predicted correction direction on the
// handle's grid from its padded residual (float) and flags

namespace les {
int net_prepare(les_net_s* n, const Dom& d, long long* generation) {
    const Level L0 = coarse(n, Level{d.nx, d.ny, d.nz});
    int rc = ensure_ws(n, L0);
    if (generation) *generation = n->ws_gen;
    return rc;
}

// the network prediction with the coarse network as one cooperative launch:
// pool (full grid) -> network (persistent) -> prolongation (full grid); the
// caller adds the line search and step.  LES_EINVAL when this device cannot
// run the cooperative launch (the caller then uses the per-layer launches).
int net_predict_persistent(les_net_s* n, const Dom& d, const float* r_padded, const uint8_t* flags, float* q_dense,
                           Scalars* sc, const int* gate, cudaStream_t s) {
    const int grid = nn::net_infer_grid();
    if (grid <= 0 || grid > kMaxInferGrid) return LES_EINVAL;
    const Level Lf{d.nx, d.ny, d.nz};
    const Level L0 = coarse(n, Lf);
    cudaStream_t keep = n->stream;
    n->stream = s;
    int rc = ensure_ws(n, L0);
    n->stream = keep;
    if (rc) return rc;
    nn::pool_padded_s(r_padded, flags, d, n->stride, n->rc, n->mc, s, gate);
    nn::NetInferArgs A{};
    A.gate = gate;
    A.sc = sc;
    for (int l = 0; l < 4; ++l) {
        const Level Ll = level(L0, l);
        A.L[l][0] = Ll.X;
        A.L[l][1] = Ll.Y;
        A.L[l][2] = Ll.Z;
    }
    A.cta = n->cta;
    A.rc = n->rc;
    A.mask = n->mc;
    A.xin = n->xin;
    for (int l = 0; l < 4; ++l) A.e[l] = n->e[l];
    for (int l = 0; l < 3; ++l) {
        A.rr[l] = n->r[l];
        A.dd[l] = n->dd[l];
    }
    for (int c = 0; c < kConvs; ++c) A.wb[c] = n->wb[c];
    A.head_w = n->w32 + n->off[kConvs];
    A.y = n->y;
    A.bar_count = n->bar;
    A.bar_gen = n->bar + 1;
    cudaError_t e = nn::net_infer_launch(A, grid, s);
    if (e == cudaSuccess) {
        nn::prolong_flags(n->y, flags, d, n->stride, q_dense, s, gate);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nfail(n, LES_ECUDA, "persistent network prediction", e);
    }
    return LES_OK;
}
int net_persistent_launches() { return 4; }     // pool, barrier reset, network, prolongation

long long net_generation(const les_net_s* n) { return n->ws_gen; }
// pooling (+ RMS and packing), the network and, with out_dense set, the
// prolongation onto the fine unknowns
int predict_impl(les_net_s* n, const Dom& d, const float* r_padded, const uint8_t* flags, float* out_dense,
                 cudaStream_t s, const int* gate, cudaEvent_t after_pool, bool fold, bool pooled) {
    nn::set_conv_engine(n->engine, n->tc_timeout);
    const Level Lf{d.nx, d.ny, d.nz};
    const Level L0 = coarse(n, Lf);
    cudaStream_t keep = n->stream;
    n->stream = s;
    int rc = ensure_ws(n, L0);
    // tcgen05 with the pooling + RMS kernel: packing and head folded into the convolutions
    const bool folded = fold && n->engine != nn::kEngineMmaSync && L0.v() <= nn::kPoolRmsMax;
    if (!rc) {
        if (L0.v() <= nn::kPoolRmsMax) {
            // pooling and RMS in one launch, the pooled mask straight into the
            // head's mask, then the packing (`pooled`: the estimate before
            // this call left them, see net_pool_target)
            n->last_launches = 0;
            if (!pooled) {
                nn::pool_rms(r_padded, flags, d, n->stride, n->rc, n->mask, n->pp_part, n->pp_count, n->dscal, s,
                             gate);
                n->last_launches = 1;
            }
            if (after_pool) cudaEventRecord(after_pool, s);      // the residual has been read
            if (!folded) {
                launch_pdl(k_pack_dense, dim3((unsigned)((L0.v() + 255) / 256)), dim3(256), 0, s,
                           (const float*)n->rc, (const float*)n->mask, (const double*)n->dscal, n->xin,
                           (size_t)L0.v(), gate);
                n->last_launches += 1;
            }
        } else {
            nn::pool_padded_s(r_padded, flags, d, n->stride, n->rc, n->mc, s, gate);
            if (after_pool) cudaEventRecord(after_pool, s);
            rc = pack_sample(n, L0, n->rc, n->mc, nullptr, nullptr, gate);
            n->last_launches = 1 + 3 + 1;
        }
    }
    if (!rc) {
        if (folded) {
            forward_tc_folded(n, L0, gate);
            n->last_launches += 7;
        } else {
            forward_fused(n, L0, gate);
            n->last_launches += 8;
        }
        if (out_dense) {
            nn::prolong_flags(n->y, flags, d, n->stride, out_dense, s, gate);
            n->last_launches += 1;
        }
        if (cudaGetLastError() != cudaSuccess) rc = LES_ECUDA;
    }
    n->stream = keep;
    return rc;
}

int net_predict(les_net_s* n, const Dom& d, const float* r_padded, const uint8_t* flags, float* out_dense,
                cudaStream_t s, const int* gate, cudaEvent_t after_pool, bool fold, bool pooled) {
    return predict_impl(n, d, r_padded, flags, out_dense, s, gate, after_pool, fold, pooled);
}
int net_predict_coarse(les_net_s* n, const Dom& d, const float* r_padded, const uint8_t* flags, cudaStream_t s,
                       const int* gate, bool pooled) {
    return predict_impl(n, d, r_padded, flags, nullptr, s, gate, nullptr, true, pooled);
}
// the buffers pool_rms fills (pooled residual, pooled mask into the head's
// mask, RMS and mask sum), for an estimate that pools in its place
bool net_pool_target(les_net_s* n, const Dom& d, EstPool* out) {
    const Level L0 = coarse(n, Level{d.nx, d.ny, d.nz});
    if ((n->stride != 4 && n->stride != 8) || L0.v() > nn::kPoolRmsMax) return false;
    if (ensure_ws(n, L0) != LES_OK) return false;
    out->rc = n->rc;
    out->mask = n->mask;
    out->scal = n->dscal;
    out->s = n->stride;
    out->xc = L0.X;
    out->yc = L0.Y;
    out->zc = L0.Z;
    return true;
}
const float* net_coarse_out(const les_net_s* n) { return n->y; }
int net_stride(const les_net_s* n) { return n->stride; }
int net_launches(const les_net_s* n) { return n->last_launches; }   // of the last net_predict
}  // namespace les

extern "C" {

int les_net_create(uint64_t seed, void* stream, les_net* out) {
    if (!out) return LES_EINVAL;
    *out = nullptr;
    les_net_s* n = new (std::nothrow) les_net_s();
    if (!n) return LES_ENOMEM;
    n->stream = (cudaStream_t)stream;
    if (nn::conv3_prepare() != 0) {
        delete n;
        return LES_ECUDA;
    }
    size_t o = 0;
    for (int c = 0; c < kConvs; ++c) {
        n->off[c] = o;
        o += (size_t)27 * kCin[c] * kCout[c];
    }
    n->off[kConvs] = o;
    n->nparam = o + kHeadC;
    // He-normal initialisation (conv0 sees 2 live input channels)
    std::vector<float> w(n->nparam);
    uint64_t ctr = 0;
    for (int c = 0; c < kConvs; ++c) {
        const double fan = 27.0 * (c == 0 ? 2 : kCin[c]);
        const double sd = std::sqrt(2.0 / fan);
        for (size_t q = n->off[c]; q < n->off[c + 1]; ++q) w[q] = (float)(sd * normal_at(seed, ctr++));
    }
    for (int q = 0; q < kHeadC; ++q) w[n->off[kConvs] + q] = (float)(std::sqrt(1.0 / kHeadC) * normal_at(seed, ctr++));
    auto get = [&](size_t bytes, void** q) -> bool {
        if (cudaMalloc(q, bytes) != cudaSuccess) return false;
        n->owned.push_back(*q);
        return cudaMemsetAsync(*q, 0, bytes, n->stream) == cudaSuccess;
    };
    bool ok = get(n->nparam * 4, (void**)&n->w32) && get(n->nparam * 4, (void**)&n->g32) &&
              get(n->nparam * 4, (void**)&n->m32) && get(n->nparam * 4, (void**)&n->v32) &&
              get(4 * kMaxInferGrid * sizeof(double), (void**)&n->cta) && get(2 * sizeof(unsigned), (void**)&n->bar) &&
              get(2 * nn::kPoolRmsMax * sizeof(double), (void**)&n->pp_part) &&
              get(sizeof(unsigned), (void**)&n->pp_count) &&
              get(kSplitFloats * sizeof(float), (void**)&n->split.part) &&
              get(kSplitCounters * sizeof(unsigned), (void**)&n->split.cnt) &&
              get(sizeof(int), (void**)&n->tc_timeout);
    n->split.part_floats = kSplitFloats;
    n->split.counters = kSplitCounters;
    for (int c = 0; ok && c < kConvs; ++c) {
        const size_t cnt = (size_t)27 * kCin[c] * kCout[c];
        ok = get(cnt * 2, (void**)&n->wb[c]) && get(cnt * 2, (void**)&n->wt[c]);
    }
    if (ok) ok = cudaMemcpyAsync(n->w32, w.data(), n->nparam * 4, cudaMemcpyHostToDevice, n->stream) == cudaSuccess;
    if (ok) {
        refresh_copies(n);
        ok = cudaStreamSynchronize(n->stream) == cudaSuccess && cudaGetLastError() == cudaSuccess;
    }
    if (!ok) {
        for (void* q : n->owned) cudaFree(q);
        delete n;
        return LES_ENOMEM;
    }
    *out = n;
    return LES_OK;
}

void les_net_destroy(les_net n) {
    if (!n) return;
    cudaStreamSynchronize(n->stream);
    free_ws(n);
    for (void* q : n->owned) cudaFree(q);
    delete n;
}

const char* les_net_last_error(les_net n) { return n ? n->err : ""; }

int les_net_num_params(les_net n, int64_t* count) {
    if (!n || !count) return LES_EINVAL;
    *count = (int64_t)n->nparam;
    return LES_OK;
}

int les_net_get_params(les_net n, float* host) {
    if (!n || !host) return LES_EINVAL;
    NCK(cudaMemcpyAsync(host, n->w32, n->nparam * 4, cudaMemcpyDeviceToHost, n->stream));
    NCK(cudaStreamSynchronize(n->stream));
    return LES_OK;
}

int les_net_set_params(les_net n, const float* host) {
    if (!n || !host) return LES_EINVAL;
    NCK(cudaMemcpyAsync(n->w32, host, n->nparam * 4, cudaMemcpyHostToDevice, n->stream));
    refresh_copies(n);
    NCK(cudaGetLastError());
    NCK(cudaStreamSynchronize(n->stream));
    n->adam_t = 0;
    NCK(cudaMemset(n->m32, 0, n->nparam * 4));
    NCK(cudaMemset(n->v32, 0, n->nparam * 4));
    return LES_OK;
}

int les_net_set_stride(les_net n, int32_t stride) {
    if (!n || (stride != 1 && stride != 2 && stride != 4 && stride != 8)) return LES_EINVAL;
    n->stride = stride;
    return LES_OK;
}

int les_net_get_stride(les_net n, int32_t* stride) {
    if (!n || !stride) return LES_EINVAL;
    *stride = n->stride;
    return LES_OK;
}

// a tcgen05 convolution of the last synchronous call gave up a bounded wait
int tc_check(les_net_s* n) {
    int t = 0;
    NCK(cudaMemcpy(&t, n->tc_timeout, sizeof(int), cudaMemcpyDeviceToHost));
    if (!t) return LES_OK;
    NCK(cudaMemset(n->tc_timeout, 0, sizeof(int)));
    return nfail(n, LES_ETIMEOUT, "a tcgen05 convolution's bounded wait timed out");
}

int les_net_set_engine(les_net n, int32_t engine) {
    if (!n || (engine != LES_NET_MMA_SYNC && engine != LES_NET_TCGEN05 && engine != LES_NET_TCGEN05_GMEM_SPLIT))
        return LES_EINVAL;
    n->engine = engine == LES_NET_TCGEN05 ? nn::kEngineTcgen05
                : engine == LES_NET_TCGEN05_GMEM_SPLIT ? nn::kEngineTcgen05Gmem
                                                       : nn::kEngineMmaSync;
    return LES_OK;
}

int les_net_get_engine(les_net n, int32_t* engine) {
    if (!n || !engine) return LES_EINVAL;
    *engine = n->engine == nn::kEngineTcgen05       ? LES_NET_TCGEN05
              : n->engine == nn::kEngineTcgen05Gmem ? LES_NET_TCGEN05_GMEM_SPLIT
                                                    : LES_NET_MMA_SYNC;
    return LES_OK;
}

int les_net_forward(les_net n, const float* d_r, const float* d_mask, float* d_y, int32_t nx, int32_t ny,
                    int32_t nz) {
    if (!n || !d_r || !d_mask || !d_y || nx < 1 || ny < 1 || nz < 1) return LES_EINVAL;
    nn::set_conv_engine(n->engine, n->tc_timeout);
    const Level Lf{nx, ny, nz};
    const Level L0 = coarse(n, Lf);
    int rc = ensure_ws(n, L0);
    if (rc) return rc;
    if ((rc = prepare_sample(n, Lf, d_r, d_mask, nullptr, 0, nullptr))) return rc;
    forward_fused(n, L0, nullptr);
    nn::prolong_dense(n->y, d_mask, d_y, nx, ny, nz, n->stride, n->stream);
    NCK(cudaGetLastError());
    NCK(cudaStreamSynchronize(n->stream));
    return tc_check(n);
}

int les_net_gradient(les_net n, const float* d_r, const float* d_mask, const float* d_t, int32_t batch, int32_t nx,
                     int32_t ny, int32_t nz, float* d_grad, double* loss) {
    if (!n || !d_r || !d_mask || !d_t || !d_grad || !loss || batch < 1 || nx < 1 || ny < 1 || nz < 1)
        return LES_EINVAL;
    nn::set_conv_engine(n->engine, n->tc_timeout);
    int rc = batch_grad(n, Level{nx, ny, nz}, d_r, d_mask, d_t, batch, loss);
    if (rc) return rc;
    NCK(cudaMemcpyAsync(d_grad, n->g32, n->nparam * 4, cudaMemcpyDeviceToDevice, n->stream));
    NCK(cudaStreamSynchronize(n->stream));
    return tc_check(n);
}

int les_net_train_step(les_net n, const float* d_r, const float* d_mask, const float* d_t, int32_t batch, int32_t nx,
                       int32_t ny, int32_t nz, float lr, double* loss) {
    if (!n || !d_r || !d_mask || !d_t || !loss || batch < 1 || nx < 1 || ny < 1 || nz < 1 || !(lr > 0))
        return LES_EINVAL;
    nn::set_conv_engine(n->engine, n->tc_timeout);
    int rc = batch_grad(n, Level{nx, ny, nz}, d_r, d_mask, d_t, batch, loss);
    if (rc) return rc;
    n->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - std::pow(b1, (float)n->adam_t), c2 = 1.f - std::pow(b2, (float)n->adam_t);
    for (int c = 0; c <= kConvs; ++c) {
        const size_t o = n->off[c], cnt = (c < kConvs ? n->off[c + 1] : n->nparam) - o;
        nn::adam(n->w32 + o, n->m32 + o, n->v32 + o, n->g32 + o, c < kConvs ? n->wb[c] : nullptr, cnt, lr, b1, b2,
                 eps, c1, c2, n->stream);
    }
    for (int c = 0; c < kConvs; ++c) nn::wflip(n->wb[c], n->wt[c], kCin[c], kCout[c], n->stream);
    NCK(cudaGetLastError());
    NCK(cudaStreamSynchronize(n->stream));
    return tc_check(n);
}

}  // extern "C"
