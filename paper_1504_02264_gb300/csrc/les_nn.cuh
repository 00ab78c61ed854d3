// Internal declarations of the learned warm-start network (not the C ABI).
#pragma once

#include <cuda_bf16.h>

#include "les_internal.cuh"

namespace les {
namespace nn {

// set the convolution kernels' dynamic shared memory limit on the current device (0 = ok)
int conv3_prepare();
// workspace of the input-channel split of small convolutions (inference):
// FP32 partial accumulators and per-tile counters (zero between launches)
struct ConvSplit {
    float* part;
    size_t part_floats;
    unsigned* cnt;
    size_t counters;
};
// How a convolution reads input voxel (gx, gy, gz) of its X x Y x Z output
// grid from its source tensor x (Xs x Ys x Zs):
//   IN_DIRECT  x[gz][gy][gx]
//   IN_UP      x[gz/2][gy/2][gx/2]               nearest upsampling of a coarser tensor
//   IN_POOL    mean of the 8 children x[2gz+c][2gy+b][2gx+a] (missing children count as
//              zero; summed in the order of the stand-alone pooling kernel, so the
//              staged values are bit-identical to pooling first)
//   IN_PACK    the network input formed from the pooled residual: channel 0 =
//              pm r / rms, channel 1 = pm, the rest 0 (pm the pooled unknown
//              fraction, rms = scale[0]; the values of the packing kernel)
enum { IN_DIRECT = 0, IN_UP = 1, IN_POOL = 2, IN_PACK = 3 };
struct ConvArgs {
    const __nv_bfloat16* x;
    const __nv_bfloat16* w;
    __nv_bfloat16* y;
    const __nv_bfloat16* skip;
    __nv_bfloat16* ysum;
    int X, Y, Z, Cin, Cout, relu, Xs, Ys, Zs;
    // split over the input-channel chunks (ks > 1): CTA kq of an output tile
    // takes chunks [kq * nch / ks, (kq + 1) * nch / ks) and leaves its FP32
    // accumulators in part; the last CTA of the tile (counter cnt[tile]) adds
    // the ks partials in the order kq = 0, 1, ... and runs the epilogue
    float* part;
    unsigned* cnt;
    int ks;
    // tcgen05 kernel: the ks CTAs of a tile run as one thread-block cluster and
    // add their partial sums over distributed shared memory (part, cnt unused)
    int cluster;
    // IN_PACK sources (level-0 volumes and the RMS)
    const float* prc;
    const float* pmask;
    const double* pscale;
    // head folded into the epilogue (head_y set; Cout == 16, one CTA holds
    // every channel of a voxel): head_y = head_mask * sum_c head_w[c] d[c],
    // d = BF16(BF16(relu(conv)) + skip) as the stand-alone head reads it, in
    // its order c = 0, 1, ...; the convolution's own outputs are not stored
    const float* head_w;
    const float* head_mask;
    float* head_y;
};

// Which tensor-core path the forward convolutions (inference, and the
// backward pass's input gradient) run on: the warp-level mma.sync kernel or
// the tcgen05 kernel (les_nn_tc.cu), whose input-channel split adds its
// partial sums in a thread-block cluster or (kEngineTcgen05Gmem) through
// global memory.  `timeout` (device int, nullable) records
// a bounded wait of the tcgen05 kernel that gave up.  Process-wide; the
// network entry points set it from the network's own choice before launching.
constexpr int kEngineMmaSync = 0, kEngineTcgen05 = 1, kEngineTcgen05Gmem = 2;
void set_conv_engine(int engine, int* timeout);
int conv3_tc_prepare();
void conv3_tc_launch(ConvArgs A, int in_mode, cudaStream_t s, const int* gate, const ConvSplit* split, int* timeout,
                     bool cluster_split);
// tcgen05 inference: the first convolution (16 input channels) reading the
// packed input straight from the pooled residual rc, the pooled mask pm and
// the RMS scale[0]; the last decoder convolution (Cout 16, nearest
// upsampling of xc, skip added) with the head folded in, writing only the
// coarse output y_head (mask pm)
void conv3_tc_fwd_packed(const float* rc, const float* pm, const double* scale, const __nv_bfloat16* w,
                         __nv_bfloat16* y, int X, int Y, int Z, int Cout, int relu, cudaStream_t s, const int* gate,
                         const ConvSplit* split);
void conv3_tc_fwd_up_head(const __nv_bfloat16* xc, const __nv_bfloat16* w, const __nv_bfloat16* skip, int X, int Y,
                          int Z, int Cin, int relu, const float* head_w, const float* pm, float* y_head, cudaStream_t s,
                          const int* gate, const ConvSplit* split);

void conv3_fwd(const __nv_bfloat16* x, const __nv_bfloat16* w, __nv_bfloat16* y, const __nv_bfloat16* skip,
               __nv_bfloat16* ysum, int X, int Y, int Z, int Cin, int Cout, int relu, cudaStream_t s,
               const int* gate = nullptr, const ConvSplit* split = nullptr);
// the same convolution reading its input through nearest upsampling of a
// coarser tensor xc (output grid X x Y x Z, xc is ceil-halved) or through 2x2x2
// mean pooling of a finer tensor xf (Xf x Yf x Zf; output is ceil-halved)
void conv3_fwd_up(const __nv_bfloat16* xc, const __nv_bfloat16* w, __nv_bfloat16* y, const __nv_bfloat16* skip,
                  __nv_bfloat16* ysum, int X, int Y, int Z, int Cin, int Cout, int relu, cudaStream_t s,
                  const int* gate = nullptr, const ConvSplit* split = nullptr);
void conv3_fwd_pool(const __nv_bfloat16* xf, const __nv_bfloat16* w, __nv_bfloat16* y, int Xf, int Yf, int Zf,
                    int Cin, int Cout, int relu, cudaStream_t s, const int* gate = nullptr,
                    const ConvSplit* split = nullptr);
void wflip(const __nv_bfloat16* w, __nv_bfloat16* wt, int Cin, int Cout, cudaStream_t s);
void conv3_wgrad(const __nv_bfloat16* x, const __nv_bfloat16* dy, float* dw, int X, int Y, int Z, int Cin, int Cout,
                 cudaStream_t s);
// `gate` (nullable): the kernels return at once while *gate != 0 (a solve's
// done flag when the inference is captured inside a CUDA graph)
void pool(const __nv_bfloat16* a, __nv_bfloat16* b, int X, int Y, int Z, int C, cudaStream_t s,
          const int* gate = nullptr);
void pool_bwd(const __nv_bfloat16* gb, __nv_bfloat16* ga, int X, int Y, int Z, int C, cudaStream_t s);
void up(const __nv_bfloat16* b, __nv_bfloat16* a, int X, int Y, int Z, int C, cudaStream_t s,
        const int* gate = nullptr);
void up_bwd(const __nv_bfloat16* ga, __nv_bfloat16* gb, int X, int Y, int Z, int C, cudaStream_t s);
void relu_bwd(const __nv_bfloat16* post, const __nv_bfloat16* g, const __nv_bfloat16* g2, __nv_bfloat16* out,
              size_t n, cudaStream_t s);
void add(const __nv_bfloat16* a, const __nv_bfloat16* b, __nv_bfloat16* out, size_t n, cudaStream_t s);
void head(const __nv_bfloat16* d, const float* w1, const float* mask, float* y, size_t nv, int C, cudaStream_t s,
          const int* gate = nullptr);
void head_bwd(const __nv_bfloat16* d, const float* w1, const float* mask, const float* gy, __nv_bfloat16* gd,
              float* dw1, size_t nv, int C, cudaStream_t s);
void pool_dense_s(const float* a, float* b, int Xf, int Yf, int Zf, int st, cudaStream_t s);
void pool_padded_s(const float* r, const uint8_t* flags, const Dom& d, int st, float* rc, float* mc, cudaStream_t s,
                   const int* gate = nullptr);
// pool_padded_s and the RMS of the pooled residual (scal[0], mask sum in
// scal[1]) in one launch; part holds 2 doubles per block (grids of at most
// kPoolRmsMax coarse voxels), counter starts at 0
constexpr size_t kPoolRmsMax = 32768;
void pool_rms(const float* r, const uint8_t* flags, const Dom& d, int st, float* rc, float* mc, double* part,
              unsigned* counter, double* scal, cudaStream_t s, const int* gate = nullptr);
void prolong_dense(const float* yc, const float* mask, float* out, int Xf, int Yf, int Zf, int st, cudaStream_t s);
void prolong_flags(const float* yc, const uint8_t* flags, const Dom& d, int st, float* out, cudaStream_t s,
                   const int* gate = nullptr);
void mse(const float* y, const float* t, const float* mask, float* g, double* loss, size_t n, double inv_n,
         cudaStream_t s);
void adam(float* w, float* m, float* v, const float* g, __nv_bfloat16* wb, size_t n, float lr, float b1, float b2,
          float eps, float c1, float c2, cudaStream_t s);
void to_bf16(const float* a, __nv_bfloat16* b, size_t n, cudaStream_t s);

// The coarse network of the solver's correction in one cooperative persistent
// launch: RMS of the pooled residual, packing, the seven convolutions (pooling
// and upsampling folded into their staging) and the head, phases separated by
// a bounded grid barrier.  Pooling before it and prolongation, line search and
// step after it are ordinary full-grid kernels.
struct NetInferArgs {
    const int* gate;                // the solve's done flag (kernel returns at once when set; nullable)
    Scalars* sc;                    // timeout record of the grid barrier
    int L[4][3];                    // level dims (X, Y, Z); level 0 = coarse grid of the network
    double* cta;                    // [2 * grid] per-CTA partial sums
    const float* rc;                // pooled residual
    const float* mask;              // pooled unknown fraction
    __nv_bfloat16* xin;
    __nv_bfloat16* e[4];
    __nv_bfloat16* rr[3];
    __nv_bfloat16* dd[3];
    const __nv_bfloat16* wb[7];
    const float* head_w;
    float* y;                       // coarse output
    unsigned* bar_count;            // grid barrier state (count zeroed before each launch)
    unsigned* bar_gen;
};
// CTAs of the persistent launch on this device (0 if a cooperative launch is
// not possible); sets the kernel's shared-memory limit on first use
int net_infer_grid();
cudaError_t net_infer_launch(const NetInferArgs& a, int grid, cudaStream_t s);

}  // namespace nn
}  // namespace les
