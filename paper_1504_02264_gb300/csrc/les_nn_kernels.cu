// Kernels of the learned SOR warm start: a small 3-D U-Net on BF16
// activations with FP32 accumulation on the tensor cores
// (mma.sync.m16n8k16 bf16), plus the elementwise pieces of its forward and
// backward pass and the Adam update.
//
// Activations are dense NDHWC: a[((z*Y + y)*X + x)*C + c], C a multiple of 16.
// Conv weights are [27][Cout][Cin] (tap-major, input channel fastest), tap =
// (dz*3 + dy)*3 + dx with offsets -1..1, zero padding outside the volume.
#include <cuda_bf16.h>

#include "les_nn.cuh"

namespace les {
namespace nn {

// ---------------------------------------------------------------------------
// 3x3x3 convolution, implicit GEMM on mma.sync.m16n8k16 (bf16 in, fp32 acc).
// CTA: 16 x 4 x 2 output voxels, 8 warps; warp w owns the 16 voxels of row
// (y = w % 4, z = w / 4) and CO output channels.  Per 16-channel input chunk
// the input halo block (18 x 6 x 4 voxels) and the chunk's weights are staged
// in shared memory; A fragments come from ldmatrix on the voxel rows, B
// fragments from ldmatrix on the [co][ci] weight rows.
// Epilogue: y = relu?(acc) (bf16), and optionally ysum = y + skip.

constexpr int TX = 16, TY = 4, TZ = 2, HX = TX + 2, HY = TY + 2, HZ = TZ + 2;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared tiles hold 16 channels (32 bytes) per row; ldmatrix reads 8
// consecutive rows, and rows r and r+4 would fall on the same banks.  The two
// 16-byte halves of a row are swapped when bit 2 of the row index is set, so
// any 8 consecutive rows hit 8 distinct bank groups.
__device__ __forceinline__ int swz(int row) { return (row >> 2) & 1; }

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t addr, uint32_t& r0, uint32_t& r1) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0, %1}, [%2];"
                 : "=r"(r0), "=r"(r1)
                 : "r"(addr));
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int bytes) {
    // bytes = 0 fills the 16 destination bytes with zeros (src is not read)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N));
}

template <int CO>
struct ConvStage {
    __nv_bfloat16 in[HZ][HY][HX][16];
    __nv_bfloat16 w[27][CO][16];
};

// Two stages in dynamic shared memory: the next 16-channel chunk (halo block
// and weights) is copied with cp.async while the tensor cores work on the
// current one; the 27 taps are unrolled.
// IN selects how the input voxel (gx, gy, gz) of the X x Y x Z output grid is
// read from the source tensor x (Xs x Ys x Zs):
//   IN_DIRECT  x[gz][gy][gx]                     (Xs = X ...)
//   IN_UP      x[gz/2][gy/2][gx/2]               nearest upsampling of a coarser tensor
//   IN_POOL    mean of the 8 children x[2gz+c][2gy+b][2gx+a] (missing children count as
//              zero; summed in the order of the stand-alone pooling kernel, so the
//              staged values are bit-identical to pooling first)
// (IN_* and ConvArgs: les_nn.cuh)

// one output tile: (bx, by) and bz = z tile + ntz * output-channel tile;
// kq: the tile's input-channel split (0 without a split)
template <int CO, int IN>
__device__ __forceinline__ void conv_tile(const ConvArgs& A, int bx, int by, int bz, ConvStage<CO>* st, int kq = 0) {
    const __nv_bfloat16* __restrict__ x = A.x;
    const __nv_bfloat16* __restrict__ w = A.w;
    __nv_bfloat16* __restrict__ y = A.y;
    const __nv_bfloat16* __restrict__ skip = A.skip;
    __nv_bfloat16* __restrict__ ysum = A.ysum;
    const int X = A.X, Y = A.Y, Z = A.Z, Cin = A.Cin, Cout = A.Cout, relu = A.relu;
    const int Xs = A.Xs, Ys = A.Ys, Zs = A.Zs;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ntz = (Z + TZ - 1) / TZ;
    const int x0 = bx * TX, y0 = by * TY, z0 = (bz % ntz) * TZ;
    const int co0 = (bz / ntz) * CO;
    const int wy = warp % TY, wz = warp / TY;
    auto stage = [&](int c0, ConvStage<CO>& S) {
        if constexpr (IN == IN_POOL) {
            // the child loads of two items at a time in flight, then their
            // averages: two memory round trips per thread instead of four
            constexpr int NQ = HZ * HY * HX * 2, PER = (NQ + 255) / 256, R = 2;
#pragma unroll
            for (int p0 = 0; p0 < PER; p0 += R) {
                uint4 ch[R][8];
                bool in[R][8];
#pragma unroll
                for (int p = 0; p < R; ++p) {
                    const int q = tid + 256 * (p0 + p);
                    const int h = q & 1, v = q >> 1;
                    const int hx = v % HX, hy = (v / HX) % HY, hz = v / (HX * HY);
                    const int gx = x0 - 1 + hx, gy = y0 - 1 + hy, gz = z0 - 1 + hz;
                    const bool ok = p0 + p < PER && q < NQ && gx >= 0 && gx < X && gy >= 0 && gy < Y && gz >= 0 &&
                                    gz < Z;
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int fx = 2 * gx + (e & 1), fy = 2 * gy + ((e >> 1) & 1), fz = 2 * gz + (e >> 2);
                        in[p][e] = ok && fx < Xs && fy < Ys && fz < Zs;
                        ch[p][e] = in[p][e] ? *reinterpret_cast<const uint4*>(
                                                  x + (((size_t)fz * Ys + fy) * Xs + fx) * Cin + c0 + 8 * h)
                                            : make_uint4(0u, 0u, 0u, 0u);
                    }
                }
#pragma unroll
                for (int p = 0; p < R; ++p) {
                    const int q = tid + 256 * (p0 + p);
                    if (p0 + p >= PER || q >= NQ) break;
                    const int h = q & 1, v = q >> 1;
                    const int hx = v % HX, hy = (v / HX) % HY, hz = v / (HX * HY);
                    float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        if (in[p][e]) {
                            const __nv_bfloat16* b = reinterpret_cast<const __nv_bfloat16*>(&ch[p][e]);
#pragma unroll
                            for (int c = 0; c < 8; ++c) a[c] += __bfloat162float(b[c]);
                        }
                    __align__(16) __nv_bfloat16 o[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c) o[c] = __float2bfloat16(0.125f * a[c]);
                    *reinterpret_cast<uint4*>(&S.in[hz][hy][hx][8 * (h ^ swz(hx))]) =
                        *reinterpret_cast<const uint4*>(o);
                }
            }
        }
        for (int q = tid; IN != IN_POOL && q < HZ * HY * HX * 2; q += 256) {
            const int h = q & 1, v = q >> 1;
            const int hx = v % HX, hy = (v / HX) % HY, hz = v / (HX * HY);
            const int gx = x0 - 1 + hx, gy = y0 - 1 + hy, gz = z0 - 1 + hz;
            const bool ok = gx >= 0 && gx < X && gy >= 0 && gy < Y && gz >= 0 && gz < Z;
            __nv_bfloat16* dst = &S.in[hz][hy][hx][8 * (h ^ swz(hx))];
            {
                const int sx = IN == IN_UP ? gx >> 1 : gx, sy = IN == IN_UP ? gy >> 1 : gy,
                          sz = IN == IN_UP ? gz >> 1 : gz;
                const __nv_bfloat16* src = ok ? x + (((size_t)sz * Ys + sy) * Xs + sx) * Cin + c0 + 8 * h : x;
                cp_async16(smem_addr(dst), src, ok ? 16 : 0);
            }
        }
        for (int q = tid; q < 27 * CO * 2; q += 256) {
            const int h = q & 1, r = q >> 1, co = r % CO, tap = r / CO;
            const bool ok = co0 + co < Cout;
            const __nv_bfloat16* src = ok ? w + ((size_t)tap * Cout + co0 + co) * Cin + c0 + 8 * h : w;
            cp_async16(smem_addr(&S.w[tap][co][8 * (h ^ swz(co))]), src, ok ? 16 : 0);
        }
        cp_async_commit();
    };
    float acc[CO / 8][4];
#pragma unroll
    for (int n = 0; n < CO / 8; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
    const int nch = Cin / 16;
    const int ks = A.ks > 1 ? A.ks : 1;
    const int cb = kq * nch / ks, ce = (kq + 1) * nch / ks;
    const int mat = lane >> 3, r8 = lane & 7;
    const int vrow = r8 + 8 * (mat & 1), khalf = mat >> 1;
    stage(16 * cb, st[0]);
    for (int c = cb; c < ce; ++c) {
        if (c + 1 < ce) {
            stage(16 * (c + 1), st[(c + 1 - cb) & 1]);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();      // (also orders the plain shared stores of IN_POOL staging)
        const ConvStage<CO>& S = st[(c - cb) & 1];
#pragma unroll
        for (int tap = 0; tap < 27; ++tap) {
            const int dx = tap % 3, dy = (tap / 3) % 3, dz = tap / 9;
            // A: rows = 16 voxels of the warp's row shifted by the tap, k = 16 channels
            uint32_t a0, a1, a2, a3;
            ldsm_x4(smem_addr(&S.in[wz + dz][wy + dy][vrow + dx][8 * (khalf ^ swz(vrow + dx))]), a0, a1, a2, a3);
#pragma unroll
            for (int n = 0; n < CO / 8; n += 2) {
                // B: two n-tiles; matrices (co rows, ci 0-7 | 8-15) of tile n and n+1
                const int co = 8 * (n + (mat >> 1)) + r8, ko = 8 * ((mat & 1) ^ swz(co));
                uint32_t b0, b1, b2, b3;
                ldsm_x4(smem_addr(&S.w[tap][co][ko]), b0, b1, b2, b3);
                mma_bf16(acc[n], a0, a1, a2, a3, b0, b1);
                mma_bf16(acc[n + 1], a0, a1, a2, a3, b2, b3);
            }
        }
        __syncthreads();
    }
    if (ks > 1) {
        // leave this split's accumulators; the tile's last CTA adds them all
        __shared__ bool conv_last;
        const size_t tile = (size_t)bx + gridDim.x * ((size_t)by + gridDim.y * (size_t)bz);
        float4* mine = reinterpret_cast<float4*>(A.part) + ((tile * ks + kq) * 256 + tid) * (CO / 8);
#pragma unroll
        for (int n = 0; n < CO / 8; ++n) mine[n] = make_float4(acc[n][0], acc[n][1], acc[n][2], acc[n][3]);
        __threadfence();
        __syncthreads();
        if (tid == 0) conv_last = atomicAdd(&A.cnt[tile], 1u) == (unsigned)(ks - 1);
        __syncthreads();
        if (!conv_last) return;
        __threadfence();
#pragma unroll
        for (int n = 0; n < CO / 8; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
        for (int k = 0; k < ks; ++k) {
            const float4* p = reinterpret_cast<const float4*>(A.part) + ((tile * ks + k) * 256 + tid) * (CO / 8);
#pragma unroll
            for (int n = 0; n < CO / 8; ++n) {
                const float4 v = __ldcg(p + n);
                acc[n][0] += v.x;
                acc[n][1] += v.y;
                acc[n][2] += v.z;
                acc[n][3] += v.w;
            }
        }
        if (tid == 0) A.cnt[tile] = 0u;
    }
    // epilogue: thread holds rows g and g+8 (voxels), columns 2*(lane%4) + {0,1}
    const int g = lane >> 2, cq = 2 * (lane & 3);
    const int gy = y0 + wy, gz = z0 + wz;
    if (gy >= Y || gz >= Z) return;
#pragma unroll
    for (int n = 0; n < CO / 8; ++n) {
        const int co = co0 + 8 * n + cq;
        if (co >= Cout) continue;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int gx = x0 + g + 8 * hh;
            if (gx >= X) continue;
            float v0 = acc[n][2 * hh], v1 = acc[n][2 * hh + 1];
            if (relu) {
                v0 = fmaxf(v0, 0.f);
                v1 = fmaxf(v1, 0.f);
            }
            const size_t o = (((size_t)gz * Y + gy) * X + gx) * Cout + co;
            __nv_bfloat162 r = __floats2bfloat162_rn(v0, v1);
            *reinterpret_cast<__nv_bfloat162*>(y + o) = r;
            if (skip) {
                const __nv_bfloat162 s = *reinterpret_cast<const __nv_bfloat162*>(skip + o);
                *reinterpret_cast<__nv_bfloat162*>(ysum + o) =
                    __floats2bfloat162_rn(__bfloat162float(r.x) + __bfloat162float(s.x),
                                          __bfloat162float(r.y) + __bfloat162float(s.y));
            }
        }
    }
}

template <int CO, int IN>
__global__ void __launch_bounds__(256) k_conv3(ConvArgs A, const int* gate) {
    pdl_wait();
    if (gate && *(volatile const int*)gate) return;      // the solve this inference serves has ended
    extern __shared__ __align__(16) unsigned char conv_smem[];
    const int ks = A.ks > 1 ? A.ks : 1;
    conv_tile<CO, IN>(A, blockIdx.x, blockIdx.y, blockIdx.z / ks, reinterpret_cast<ConvStage<CO>*>(conv_smem),
                      blockIdx.z % ks);
}

template <int CO, int IN>
static cudaError_t allow_conv() {
    return cudaFuncSetAttribute(k_conv3<CO, IN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(2 * sizeof(ConvStage<CO>)));
}

int conv3_prepare() {
    if (conv3_tc_prepare() != 0) return -1;
    cudaError_t e = cudaSuccess, x;
    if ((x = allow_conv<32, IN_DIRECT>()) != cudaSuccess) e = x;
    if ((x = allow_conv<16, IN_DIRECT>()) != cudaSuccess) e = x;
    if ((x = allow_conv<32, IN_UP>()) != cudaSuccess) e = x;
    if ((x = allow_conv<16, IN_UP>()) != cudaSuccess) e = x;
    if ((x = allow_conv<32, IN_POOL>()) != cudaSuccess) e = x;
    if ((x = allow_conv<16, IN_POOL>()) != cudaSuccess) e = x;
    return e == cudaSuccess ? 0 : -1;
}

int g_conv_engine = kEngineTcgen05;
int* g_conv_timeout = nullptr;

void set_conv_engine(int engine, int* timeout) {
    g_conv_engine = engine;
    g_conv_timeout = timeout;
}

template <int IN>
static void conv3_launch(const __nv_bfloat16* x, const __nv_bfloat16* w, __nv_bfloat16* y, const __nv_bfloat16* skip,
                         __nv_bfloat16* ysum, int X, int Y, int Z, int Cin, int Cout, int relu, cudaStream_t s,
                         const int* gate, int Xs, int Ys, int Zs, const ConvSplit* split) {
    if (g_conv_engine != kEngineMmaSync) {
        const ConvArgs A{x, w, y, skip, ysum, X, Y, Z, Cin, Cout, relu, Xs, Ys, Zs, nullptr, nullptr, 1};
        conv3_tc_launch(A, IN, s, gate, split, g_conv_timeout, g_conv_engine == kEngineTcgen05);
        return;
    }
    // 32 output channels per CTA when the grid fills the GPU, else 16 (twice
    // the CTAs, half the weights staged per CTA: small levels are latency-bound)
    const int ntz = (Z + TZ - 1) / TZ;
    const long long tiles = (long long)((X + TX - 1) / TX) * ((Y + TY - 1) / TY) * ntz;
    const int co = (Cout >= 32 && tiles * (Cout / 32) >= 2 * 152) ? 32 : 16;
    dim3 grid((X + TX - 1) / TX, (Y + TY - 1) / TY, ntz * ((Cout + co - 1) / co));
    // with a split workspace, small grids (few CTAs, latency-bound) split the
    // input-channel chunks over more CTAs, up to about two per SM
    int ks = 1;
    if (split && co == 16) {
        const long long ctas = (long long)grid.x * grid.y * grid.z;
        const int nch = Cin / 16;
        while (nch % (2 * ks) == 0 && ctas * 2 * ks <= 2 * 152 &&
               (size_t)ctas * 2 * ks * 256 * (co / 2) <= split->part_floats && (size_t)ctas <= split->counters)
            ks *= 2;
        grid.z *= ks;
    }
    const ConvArgs A{x, w, y, skip, ysum, X, Y, Z, Cin, Cout, relu, Xs, Ys, Zs,
                     ks > 1 ? split->part : nullptr, ks > 1 ? split->cnt : nullptr, ks};
    if (co == 32)
        launch_pdl(k_conv3<32, IN>, grid, dim3(256), 2 * sizeof(ConvStage<32>), s, A, gate);
    else
        launch_pdl(k_conv3<16, IN>, grid, dim3(256), 2 * sizeof(ConvStage<16>), s, A, gate);
}

void conv3_fwd(const __nv_bfloat16* x, const __nv_bfloat16* w, __nv_bfloat16* y, const __nv_bfloat16* skip,
               __nv_bfloat16* ysum, int X, int Y, int Z, int Cin, int Cout, int relu, cudaStream_t s,
               const int* gate, const ConvSplit* split) {
    conv3_launch<IN_DIRECT>(x, w, y, skip, ysum, X, Y, Z, Cin, Cout, relu, s, gate, X, Y, Z, split);
}

void conv3_fwd_up(const __nv_bfloat16* xc, const __nv_bfloat16* w, __nv_bfloat16* y, const __nv_bfloat16* skip,
                  __nv_bfloat16* ysum, int X, int Y, int Z, int Cin, int Cout, int relu, cudaStream_t s,
                  const int* gate, const ConvSplit* split) {
    conv3_launch<IN_UP>(xc, w, y, skip, ysum, X, Y, Z, Cin, Cout, relu, s, gate, (X + 1) / 2, (Y + 1) / 2,
                        (Z + 1) / 2, split);
}

void conv3_tc_fwd_packed(const float* rc, const float* pm, const double* scale, const __nv_bfloat16* w,
                         __nv_bfloat16* y, int X, int Y, int Z, int Cout, int relu, cudaStream_t s, const int* gate,
                         const ConvSplit* split) {
    ConvArgs A{nullptr, w, y, nullptr, nullptr, X, Y, Z, 16, Cout, relu, X, Y, Z, nullptr, nullptr, 1};
    A.prc = rc;
    A.pmask = pm;
    A.pscale = scale;
    conv3_tc_launch(A, IN_PACK, s, gate, split, g_conv_timeout, g_conv_engine == kEngineTcgen05);
}

void conv3_tc_fwd_up_head(const __nv_bfloat16* xc, const __nv_bfloat16* w, const __nv_bfloat16* skip, int X, int Y,
                          int Z, int Cin, int relu, const float* head_w, const float* pm, float* y_head, cudaStream_t s,
                          const int* gate, const ConvSplit* split) {
    ConvArgs A{xc, w, nullptr, skip, nullptr, X, Y, Z, Cin, 16, relu, (X + 1) / 2, (Y + 1) / 2, (Z + 1) / 2,
               nullptr, nullptr, 1};
    A.head_w = head_w;
    A.head_mask = pm;
    A.head_y = y_head;
    conv3_tc_launch(A, IN_UP, s, gate, split, g_conv_timeout, g_conv_engine == kEngineTcgen05);
}

void conv3_fwd_pool(const __nv_bfloat16* xf, const __nv_bfloat16* w, __nv_bfloat16* y, int Xf, int Yf, int Zf,
                    int Cin, int Cout, int relu, cudaStream_t s, const int* gate, const ConvSplit* split) {
    conv3_launch<IN_POOL>(xf, w, y, nullptr, nullptr, (Xf + 1) / 2, (Yf + 1) / 2, (Zf + 1) / 2, Cin, Cout, relu, s,
                          gate, Xf, Yf, Zf, split);
}

// dgrad weights: W'[tap][ci][co] = W[26 - tap][co][ci] (flipped taps, swapped roles)
__global__ void k_wflip(const __nv_bfloat16* w, __nv_bfloat16* wt, int Cin, int Cout) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 27 * Cin * Cout) return;
    const int co = q % Cout, ci = (q / Cout) % Cin, tap = q / (Cout * Cin);
    wt[((size_t)tap * Cin + ci) * Cout + co] = w[((size_t)(26 - tap) * Cout + co) * Cin + ci];
}

void wflip(const __nv_bfloat16* w, __nv_bfloat16* wt, int Cin, int Cout, cudaStream_t s) {
    const int n = 27 * Cin * Cout;
    k_wflip<<<(n + 255) / 256, 256, 0, s>>>(w, wt, Cin, Cout);
}

// ---------------------------------------------------------------------------
// Weight gradient: dW[tap][co][ci] += sum_v dY[v][co] * X[v + off(tap)][ci].
// mma with M = co (16), N = ci (8), K = 16 voxels of one row; A = dY^T and
// B = X_tap loaded with ldmatrix.trans from the [voxel][channel] tiles.  A CTA
// walks `tiles` voxel blocks of one (co, ci) 16 x 16 pair; warp w owns taps
// w, w+8, w+16, w+24.  Partial sums go to the FP32 gradient with atomics.
__global__ void __launch_bounds__(256)
k_conv3_wgrad(const __nv_bfloat16* __restrict__ x, const __nv_bfloat16* __restrict__ dy, float* __restrict__ dw,
              int X, int Y, int Z, int Cin, int Cout, int tiles) {
    __shared__ __align__(16) __nv_bfloat16 sIn[HZ][HY][HX][16];
    __shared__ __align__(16) __nv_bfloat16 sG[TZ][TY][TX][16];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int co0 = blockIdx.y * 16, ci0 = blockIdx.z * 16;
    const int nbx = (X + TX - 1) / TX, nby = (Y + TY - 1) / TY, nbz = (Z + TZ - 1) / TZ;
    const int ntile = nbx * nby * nbz;
    float acc[4][2][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int n = 0; n < 2; ++n) acc[a][n][0] = acc[a][n][1] = acc[a][n][2] = acc[a][n][3] = 0.f;
    const int mat = lane >> 3, r8 = lane & 7;
    for (int t = blockIdx.x * tiles; t < min(ntile, (blockIdx.x + 1) * tiles); ++t) {
        const int bx = t % nbx, by = (t / nbx) % nby, bz = t / (nbx * nby);
        const int x0 = bx * TX, y0 = by * TY, z0 = bz * TZ;
        for (int q = tid; q < HZ * HY * HX * 2; q += 256) {
            const int h = q & 1, v = q >> 1;
            const int hx = v % HX, hy = (v / HX) % HY, hz = v / (HX * HY);
            const int gx = x0 - 1 + hx, gy = y0 - 1 + hy, gz = z0 - 1 + hz;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (gx >= 0 && gx < X && gy >= 0 && gy < Y && gz >= 0 && gz < Z)
                val = *reinterpret_cast<const uint4*>(x + (((size_t)gz * Y + gy) * X + gx) * Cin + ci0 + 8 * h);
            *reinterpret_cast<uint4*>(&sIn[hz][hy][hx][8 * (h ^ swz(hx))]) = val;
        }
        for (int q = tid; q < TZ * TY * TX * 2; q += 256) {
            const int h = q & 1, v = q >> 1;
            const int lx = v % TX, ly = (v / TX) % TY, lz = v / (TX * TY);
            const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (gx < X && gy < Y && gz < Z)
                val = *reinterpret_cast<const uint4*>(dy + (((size_t)gz * Y + gy) * X + gx) * Cout + co0 + 8 * h);
            *reinterpret_cast<uint4*>(&sG[lz][ly][lx][8 * (h ^ swz(lx))]) = val;
        }
        __syncthreads();
        for (int row = 0; row < TY * TZ; ++row) {
            const int ry = row % TY, rz = row / TY;
            // A = dY^T (m = co 16, k = 16 voxels): transposed 8x8 blocks of sG[voxel][co]
            // matrices: (co 0-7, v 0-7), (co 8-15, v 0-7), (co 0-7, v 8-15), (co 8-15, v 8-15)
            uint32_t a0, a1, a2, a3;
            {
                const int v = r8 + 8 * (mat >> 1), c = 8 * ((mat & 1) ^ swz(v));
                ldsm_x4_t(smem_addr(&sG[rz][ry][v][c]), a0, a1, a2, a3);
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int tap = warp + 8 * a;
                if (tap >= 27) break;
                const int dx = tap % 3, dyy = (tap / 3) % 3, dz = tap / 9;
                // B = X_tap (k = 16 voxels, n = 8 ci) per n-tile: transposed blocks of sIn[voxel][ci]
#pragma unroll
                for (int n = 0; n < 2; ++n) {
                    uint32_t b0, b1;
                    const int v = r8 + 8 * (mat & 1);
                    ldsm_x2_t(smem_addr(&sIn[rz + dz][ry + dyy][v + dx][8 * (n ^ swz(v + dx))]), b0, b1);
                    mma_bf16(acc[a][n], a0, a1, a2, a3, b0, b1);
                }
            }
        }
        __syncthreads();
    }
    // acc[a][n]: rows co = g, g+8 ; cols ci = 8n + 2(lane%4) + {0,1}
    const int g = lane >> 2, cq = 2 * (lane & 3);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int tap = warp + 8 * a;
        if (tap >= 27) break;
#pragma unroll
        for (int n = 0; n < 2; ++n)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int co = co0 + g + 8 * (e >> 1), ci = ci0 + 8 * n + cq + (e & 1);
                atomicAdd(&dw[((size_t)tap * Cout + co) * Cin + ci], acc[a][n][e]);
            }
    }
}

void conv3_wgrad(const __nv_bfloat16* x, const __nv_bfloat16* dy, float* dw, int X, int Y, int Z, int Cin, int Cout,
                 cudaStream_t s) {
    const int ntile = ((X + TX - 1) / TX) * ((Y + TY - 1) / TY) * ((Z + TZ - 1) / TZ);
    const int tiles = ntile < 32 ? 1 : 32;
    dim3 grid((ntile + tiles - 1) / tiles, Cout / 16, Cin / 16);
    k_conv3_wgrad<<<grid, 256, 0, s>>>(x, dy, dw, X, Y, Z, Cin, Cout, tiles);
}

// ---------------------------------------------------------------------------
// elementwise pieces

// 2x2x2 average pool (children outside the fine grid count as zero)
__global__ void k_pool(const __nv_bfloat16* a, __nv_bfloat16* b, int X, int Y, int Z, int C, const int* gate) {
    if (gate && *(volatile const int*)gate) return;
    const int Xc = (X + 1) / 2, Yc = (Y + 1) / 2, Zc = (Z + 1) / 2;
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (size_t)Xc * Yc * Zc * C) return;
    const int c = q % C;
    size_t v = q / C;
    const int x = v % Xc, yv = (v / Xc) % Yc, z = v / ((size_t)Xc * Yc);
    float s = 0.f;
    for (int e = 0; e < 8; ++e) {
        const int fx = 2 * x + (e & 1), fy = 2 * yv + ((e >> 1) & 1), fz = 2 * z + (e >> 2);
        if (fx < X && fy < Y && fz < Z) s += __bfloat162float(a[(((size_t)fz * Y + fy) * X + fx) * C + c]);
    }
    b[q] = __float2bfloat16(0.125f * s);
}
// adjoint: each fine voxel receives 1/8 of its parent's gradient
__global__ void k_pool_bwd(const __nv_bfloat16* gb, __nv_bfloat16* ga, int X, int Y, int Z, int C) {
    const int Xc = (X + 1) / 2, Yc = (Y + 1) / 2;
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (size_t)X * Y * Z * C) return;
    const int c = q % C;
    size_t v = q / C;
    const int x = v % X, yv = (v / X) % Y, z = v / ((size_t)X * Y);
    ga[q] = __float2bfloat16(0.125f * __bfloat162float(gb[(((size_t)(z / 2) * Yc + yv / 2) * Xc + x / 2) * C + c]));
}
// nearest upsample: fine voxel takes its parent's value
__global__ void k_up(const __nv_bfloat16* b, __nv_bfloat16* a, int X, int Y, int Z, int C, const int* gate) {
    if (gate && *(volatile const int*)gate) return;
    const int Xc = (X + 1) / 2, Yc = (Y + 1) / 2;
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (size_t)X * Y * Z * C) return;
    const int c = q % C;
    size_t v = q / C;
    const int x = v % X, yv = (v / X) % Y, z = v / ((size_t)X * Y);
    a[q] = b[(((size_t)(z / 2) * Yc + yv / 2) * Xc + x / 2) * C + c];
}
// adjoint: parent sums its (existing) children
__global__ void k_up_bwd(const __nv_bfloat16* ga, __nv_bfloat16* gb, int X, int Y, int Z, int C) {
    const int Xc = (X + 1) / 2, Yc = (Y + 1) / 2, Zc = (Z + 1) / 2;
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (size_t)Xc * Yc * Zc * C) return;
    const int c = q % C;
    size_t v = q / C;
    const int x = v % Xc, yv = (v / Xc) % Yc, z = v / ((size_t)Xc * Yc);
    float s = 0.f;
    for (int e = 0; e < 8; ++e) {
        const int fx = 2 * x + (e & 1), fy = 2 * yv + ((e >> 1) & 1), fz = 2 * z + (e >> 2);
        if (fx < X && fy < Y && fz < Z) s += __bfloat162float(ga[(((size_t)fz * Y + fy) * X + fx) * C + c]);
    }
    gb[q] = __float2bfloat16(s);
}
// g_pre = g_post * (post > 0); optional extra gradient added first (skip branch)
__global__ void k_relu_bwd(const __nv_bfloat16* post, const __nv_bfloat16* g, const __nv_bfloat16* g2,
                           __nv_bfloat16* out, size_t n) {
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    float v = __bfloat162float(g[q]) + (g2 ? __bfloat162float(g2[q]) : 0.f);
    out[q] = __float2bfloat16(__bfloat162float(post[q]) > 0.f ? v : 0.f);
}
__global__ void k_add(const __nv_bfloat16* a, const __nv_bfloat16* b, __nv_bfloat16* out, size_t n) {
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    out[q] = __float2bfloat16(__bfloat162float(a[q]) + __bfloat162float(b[q]));
}

// head: y[v] = mask[v] * sum_c w1[c] * d[v][c]  (FP32 output)
__global__ void k_head(const __nv_bfloat16* d, const float* w1, const float* mask, float* y, size_t nv, int C,
                       const int* gate) {
    pdl_wait();
    if (gate && *(volatile const int*)gate) return;
    const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    float s = 0.f;
    for (int c = 0; c < C; ++c) s += w1[c] * __bfloat162float(d[v * C + c]);
    y[v] = mask[v] * s;
}
// head backward: gd[v][c] = gy[v]*mask[v]*w1[c]; dw1[c] += sum_v gy[v]*mask[v]*d[v][c]
__global__ void k_head_bwd(const __nv_bfloat16* d, const float* w1, const float* mask, const float* gy,
                           __nv_bfloat16* gd, float* dw1, size_t nv, int C) {
    __shared__ float part[16][17];
    const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    float loc[16];
    for (int c = 0; c < 16; ++c) loc[c] = 0.f;
    if (v < nv) {
        const float gm = gy[v] * mask[v];
        for (int c = 0; c < C; ++c) {
            gd[v * C + c] = __float2bfloat16(gm * w1[c]);
            loc[c] = gm * __bfloat162float(d[v * C + c]);
        }
    }
    for (int c = 0; c < 16; ++c)
        for (int o = 16; o > 0; o >>= 1) loc[c] += __shfl_down_sync(0xffffffffu, loc[c], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int c = 0; c < 16; ++c) part[warp][c] = loc[c];
    __syncthreads();
    if (threadIdx.x < C) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w][threadIdx.x];
        atomicAdd(&dw1[threadIdx.x], s);
    }
}

// ---------------------------------------------------------------------------
// input stride s (the network runs on the grid coarsened s times per axis):
// coarse value = sum of the existing fine children / s^3

// dense fine [Zf][Yf][Xf] -> dense coarse
__global__ void k_pool_dense_s(const float* a, float* b, int Xf, int Yf, int Zf, int s) {
    const int Xc = (Xf + s - 1) / s, Yc = (Yf + s - 1) / s, Zc = (Zf + s - 1) / s;
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (size_t)Xc * Yc * Zc) return;
    const int x = q % Xc, y = (q / Xc) % Yc, z = q / ((size_t)Xc * Yc);
    float acc = 0.f;
    for (int dz = 0; dz < s; ++dz)
        for (int dy = 0; dy < s; ++dy)
            for (int dx = 0; dx < s; ++dx) {
                const int fx = x * s + dx, fy = y * s + dy, fz = z * s + dz;
                if (fx < Xf && fy < Yf && fz < Zf) acc += a[((size_t)fz * Yf + fy) * Xf + fx];
            }
    b[q] = acc / (float)(s * s * s);
}

// the solver's padded residual (unknowns only) and unknown mask -> dense
// coarse.  Block (32, S, SZ): thread (tx, ty, tz) sums the S fine cells of
// one fine row (y = cy*S + ty, z = cz*S + tz [+ SZ ...]) under coarse cell
// cx = blockIdx.x*32 + tx, then the block adds the rows in shared memory
// (fixed order: deterministic).
template <int S>
__global__ void k_pool_padded_s(const float* r, const uint8_t* flags, Dom d, float* rc, float* mc, const int* gate) {
    constexpr int SZ = S < 4 ? S : 4;
    __shared__ float sr[SZ][S][32], sm[SZ][S][32];
    if (gate && *(volatile const int*)gate) return;
    const int Xc = (d.nx + S - 1) / S, Yc = (d.ny + S - 1) / S;
    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    const int cx = blockIdx.x * 32 + tx, cy = blockIdx.y, cz = blockIdx.z;
    float ar = 0.f, am = 0.f;
    const int fy = cy * S + ty;
    if (cx < Xc && fy < d.ny) {
#pragma unroll
        for (int zz = 0; zz < S; zz += SZ) {
            const int fz = cz * S + tz + zz;
            if (fz >= d.nz) break;
            const long long row = d.at(1, fy + 1, fz + 1) + (long long)cx * S;
            // the row's flags and residuals are read first, unconditionally
            // (past the grid's last cell the padded array holds the ghost
            // column and the next row), then summed in order
            uint8_t fl[S];
            float rv[S];
#pragma unroll
            for (int dx = 0; dx < S; ++dx) {
                fl[dx] = flags[row + dx];
                rv[dx] = r[row + dx];
            }
#pragma unroll
            for (int dx = 0; dx < S; ++dx)
                if (cx * S + dx < d.nx && (fl[dx] & F_UNK)) {
                    ar += rv[dx];
                    am += 1.f;
                }
        }
    }
    sr[tz][ty][tx] = ar;
    sm[tz][ty][tx] = am;
    __syncthreads();
    if (ty == 0 && tz == 0 && cx < Xc) {
        float tr = 0.f, tm = 0.f;
#pragma unroll
        for (int a = 0; a < SZ; ++a)
#pragma unroll
            for (int b = 0; b < S; ++b) {
                tr += sr[a][b][tx];
                tm += sm[a][b][tx];
            }
        const float inv = 1.f / (float)(S * S * S);
        const int q = (cz * Yc + cy) * Xc + cx;
        rc[q] = tr * inv;
        mc[q] = tm * inv;
    }
}

// Pooling and the RMS of the inference input in one launch: every block
// pools its coarse cells as k_pool_padded_s does (same sums, same order) and
// leaves its partial sums of m r^2 and m (FP64); the last block to finish adds
// the partials in block order (fixed: deterministic) and stores the RMS and
// the mask sum, as k_rms and k_rms_final do.
template <int S>
__global__ void k_pool_rms(const float* r, const uint8_t* flags, Dom d, float* rc, float* mc, double* part,
                           unsigned* counter, double* scal, const int* gate) {
    constexpr int SZ = S < 4 ? S : 4;
    __shared__ float sr[SZ][S][32], sm[SZ][S][32];
    __shared__ bool last;
    pdl_wait();
    // the next kernel (the first convolution) may launch and copy its weights
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (gate && *(volatile const int*)gate) return;
    const int Xc = (d.nx + S - 1) / S, Yc = (d.ny + S - 1) / S;
    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    const int tid = tx + 32 * (ty + S * tz);
    const int cx = blockIdx.x * 32 + tx, cy = blockIdx.y, cz = blockIdx.z;
    float ar = 0.f, am = 0.f;
    const int fy = cy * S + ty;
    if (cx < Xc && fy < d.ny) {
#pragma unroll
        for (int zz = 0; zz < S; zz += SZ) {
            const int fz = cz * S + tz + zz;
            if (fz >= d.nz) break;
            const long long row = d.at(1, fy + 1, fz + 1) + (long long)cx * S;
#pragma unroll
            for (int dx = 0; dx < S; ++dx)
                if (cx * S + dx < d.nx && (flags[row + dx] & F_UNK)) {
                    ar += r[row + dx];
                    am += 1.f;
                }
        }
    }
    sr[tz][ty][tx] = ar;
    sm[tz][ty][tx] = am;
    __syncthreads();
    const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
    if (ty == 0 && tz == 0) {
        double a = 0.0, m = 0.0;
        if (cx < Xc) {
            float tr = 0.f, tm = 0.f;
#pragma unroll
            for (int p = 0; p < SZ; ++p)
#pragma unroll
                for (int q = 0; q < S; ++q) {
                    tr += sr[p][q][tx];
                    tm += sm[p][q][tx];
                }
            const float inv = 1.f / (float)(S * S * S);
            const int v = (cz * Yc + cy) * Xc + cx;
            const float vr = tr * inv, vm = tm * inv;
            rc[v] = vr;
            mc[v] = vm;
            a = (double)vm * (double)vr * (double)vr;
            m = (double)vm;
        }
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            m += __shfl_down_sync(0xffffffffu, m, o);
        }
        __threadfence();
        if (tx == 0) {
            const unsigned b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
            part[2 * b] = a;
            part[2 * b + 1] = m;
            __threadfence();
            last = atomicAdd(counter, 1u) == nb - 1;
        }
    }
    __syncthreads();
    if (!last || tid >= 32) return;
    // one warp adds the partials: FP64 arithmetic is narrow on this part, so
    // a whole-block tree would queue on it
    __threadfence();
    double a = 0.0, m = 0.0;
    for (unsigned q = tid; q < nb; q += 32) {
        a += __ldcg(&part[2 * q]);
        m += __ldcg(&part[2 * q + 1]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        m += __shfl_down_sync(0xffffffffu, m, o);
    }
    if (tid == 0) {
        scal[0] = m > 0.0 ? sqrt(a / m) : 0.0;
        scal[1] = m;
        *counter = 0u;
    }
}

// trilinear prolongation of a coarse cell-centred field to the fine cells
// (the weights of prolong_w: fine centre f at coarse coordinate (f + 1/2)/s - 1/2,
// clamped to the first / last coarse centre)
__device__ __forceinline__ void lin_w(int f, int s, int C, int& c0, float& w) { prolong_w(f, s, C, c0, w); }
__device__ __forceinline__ float trilinear(const float* y, int Xc, int Yc, int Zc, int s, int fx, int fy, int fz) {
    int x0, y0, z0;
    float wx, wy, wz;
    lin_w(fx, s, Xc, x0, wx);
    lin_w(fy, s, Yc, y0, wy);
    lin_w(fz, s, Zc, z0, wz);
    const int x1 = min(x0 + 1, Xc - 1), y1 = min(y0 + 1, Yc - 1), z1 = min(z0 + 1, Zc - 1);
    auto at = [&](int a, int b, int c) { return y[((size_t)c * Yc + b) * Xc + a]; };
    const float c00 = (1.f - wx) * at(x0, y0, z0) + wx * at(x1, y0, z0);
    const float c10 = (1.f - wx) * at(x0, y1, z0) + wx * at(x1, y1, z0);
    const float c01 = (1.f - wx) * at(x0, y0, z1) + wx * at(x1, y0, z1);
    const float c11 = (1.f - wx) * at(x0, y1, z1) + wx * at(x1, y1, z1);
    const float c0 = (1.f - wy) * c00 + wy * c10, c1 = (1.f - wy) * c01 + wy * c11;
    return (1.f - wz) * c0 + wz * c1;
}
// dense fine output with a dense fine mask
__global__ void k_prolong_dense(const float* yc, const float* mask, float* out, int Xf, int Yf, int Zf, int s) {
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (size_t)Xf * Yf * Zf) return;
    const int x = q % Xf, y = (q / Xf) % Yf, z = q / ((size_t)Xf * Yf);
    const int Xc = (Xf + s - 1) / s, Yc = (Yf + s - 1) / s, Zc = (Zf + s - 1) / s;
    out[q] = mask[q] * trilinear(yc, Xc, Yc, Zc, s, x, y, z);
}
// dense fine output on the solver's unknowns: a CTA takes a 32 x 8 tile of
// fine columns over kProlongKC planes (few CTAs: with one CTA per fine row
// the launch, not the work, bounded the kernel); each fine cell interpolates
// the (y, z)-interpolated coarse columns x0 and x1, then in x
constexpr int kProlongKC = 8;
template <int S>
__global__ void __launch_bounds__(256) k_prolong_flags(const float* yc, const uint8_t* flags, Dom d, float* out,
                                                       const int* gate) {
    pdl_wait();
    if (gate && *(volatile const int*)gate) return;
    const int Xc = (d.nx + S - 1) / S, Yc = (d.ny + S - 1) / S, Zc = (d.nz + S - 1) / S;
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    const int zb = blockIdx.z * kProlongKC, ze = min(zb + kProlongKC, d.nz);
    if (x >= d.nx || y >= d.ny) return;
    int y0, x0;
    float wy, wx;
    lin_w(y, S, Yc, y0, wy);
    lin_w(x, S, Xc, x0, wx);
    const int y1 = min(y0 + 1, Yc - 1), x1 = min(x0 + 1, Xc - 1);
    for (int z = zb; z < ze; ++z) {
        int z0;
        float wz;
        lin_w(z, S, Zc, z0, wz);
        const int z1 = min(z0 + 1, Zc - 1);
        const float v0 = prolong_col(yc, Xc, Yc, x0, y0, y1, wy, z0, z1, wz);
        const float v1 = prolong_col(yc, Xc, Yc, x1, y0, y1, wy, z0, z1, wz);
        const long long row = d.at(1, y + 1, z + 1);
        out[((size_t)z * d.ny + y) * d.nx + x] = (flags[row + x] & F_UNK) ? prolong_mix(v0, v1, wx) : 0.f;
    }
}

// training loss 1/n * sum mask (y - t)^2 and its gradient
__global__ void k_mse(const float* y, const float* t, const float* mask, float* g, double* loss, size_t n, double inv_n) {
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double e2 = 0.0;
    if (q < n) {
        const float e = mask[q] * (y[q] - t[q]);
        g[q] = (float)(2.0 * inv_n) * e;
        e2 = (double)e * e;
    }
    for (int o = 16; o > 0; o >>= 1) e2 += __shfl_down_sync(0xffffffffu, e2, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, e2 * inv_n);
}

// Adam on FP32 master weights, refreshing the BF16 copy
__global__ void k_adam(float* w, float* m, float* v, const float* g, __nv_bfloat16* wb, size_t n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.f - b1) * gq;
    const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    const float wq = w[q] - lr * (mq / c1) / (sqrtf(vq / c2) + eps);
    w[q] = wq;
    if (wb) wb[q] = __float2bfloat16(wq);
}

__global__ void k_to_bf16(const float* a, __nv_bfloat16* b, size_t n) {
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) b[q] = __float2bfloat16(a[q]);
}

static unsigned blocks_for(size_t n) { return (unsigned)((n + 255) / 256); }

void pool(const __nv_bfloat16* a, __nv_bfloat16* b, int X, int Y, int Z, int C, cudaStream_t s, const int* gate) {
    k_pool<<<blocks_for((size_t)((X + 1) / 2) * ((Y + 1) / 2) * ((Z + 1) / 2) * C), 256, 0, s>>>(a, b, X, Y, Z, C,
                                                                                                  gate);
}
void pool_bwd(const __nv_bfloat16* gb, __nv_bfloat16* ga, int X, int Y, int Z, int C, cudaStream_t s) {
    k_pool_bwd<<<blocks_for((size_t)X * Y * Z * C), 256, 0, s>>>(gb, ga, X, Y, Z, C);
}
void up(const __nv_bfloat16* b, __nv_bfloat16* a, int X, int Y, int Z, int C, cudaStream_t s, const int* gate) {
    k_up<<<blocks_for((size_t)X * Y * Z * C), 256, 0, s>>>(b, a, X, Y, Z, C, gate);
}
void up_bwd(const __nv_bfloat16* ga, __nv_bfloat16* gb, int X, int Y, int Z, int C, cudaStream_t s) {
    k_up_bwd<<<blocks_for((size_t)((X + 1) / 2) * ((Y + 1) / 2) * ((Z + 1) / 2) * C), 256, 0, s>>>(ga, gb, X, Y, Z, C);
}
void relu_bwd(const __nv_bfloat16* post, const __nv_bfloat16* g, const __nv_bfloat16* g2, __nv_bfloat16* out,
              size_t n, cudaStream_t s) {
    k_relu_bwd<<<blocks_for(n), 256, 0, s>>>(post, g, g2, out, n);
}
void add(const __nv_bfloat16* a, const __nv_bfloat16* b, __nv_bfloat16* out, size_t n, cudaStream_t s) {
    k_add<<<blocks_for(n), 256, 0, s>>>(a, b, out, n);
}
void head(const __nv_bfloat16* d, const float* w1, const float* mask, float* y, size_t nv, int C, cudaStream_t s,
          const int* gate) {
    launch_pdl(k_head, dim3(blocks_for(nv)), dim3(256), 0, s, d, w1, mask, y, nv, C, gate);
}
void head_bwd(const __nv_bfloat16* d, const float* w1, const float* mask, const float* gy, __nv_bfloat16* gd,
              float* dw1, size_t nv, int C, cudaStream_t s) {
    k_head_bwd<<<blocks_for(nv), 256, 0, s>>>(d, w1, mask, gy, gd, dw1, nv, C);
}
void pool_dense_s(const float* a, float* b, int Xf, int Yf, int Zf, int st, cudaStream_t s) {
    const size_t n = (size_t)((Xf + st - 1) / st) * ((Yf + st - 1) / st) * ((Zf + st - 1) / st);
    k_pool_dense_s<<<blocks_for(n), 256, 0, s>>>(a, b, Xf, Yf, Zf, st);
}
void pool_padded_s(const float* r, const uint8_t* flags, const Dom& d, int st, float* rc, float* mc, cudaStream_t s,
                   const int* gate) {
    const int Xc = (d.nx + st - 1) / st, Yc = (d.ny + st - 1) / st, Zc = (d.nz + st - 1) / st;
    const dim3 grid((Xc + 31) / 32, Yc, Zc);
    switch (st) {
        case 1: k_pool_padded_s<1><<<grid, dim3(32, 1, 1), 0, s>>>(r, flags, d, rc, mc, gate); break;
        case 2: k_pool_padded_s<2><<<grid, dim3(32, 2, 2), 0, s>>>(r, flags, d, rc, mc, gate); break;
        case 4: k_pool_padded_s<4><<<grid, dim3(32, 4, 4), 0, s>>>(r, flags, d, rc, mc, gate); break;
        default: k_pool_padded_s<8><<<grid, dim3(32, 8, 4), 0, s>>>(r, flags, d, rc, mc, gate); break;
    }
}
void pool_rms(const float* r, const uint8_t* flags, const Dom& d, int st, float* rc, float* mc, double* part,
              unsigned* counter, double* scal, cudaStream_t s, const int* gate) {
    const int Xc = (d.nx + st - 1) / st, Yc = (d.ny + st - 1) / st, Zc = (d.nz + st - 1) / st;
    const dim3 grid((Xc + 31) / 32, Yc, Zc);
    switch (st) {
        case 1: launch_pdl(k_pool_rms<1>, grid, dim3(32, 1, 1), 0, s, r, flags, d, rc, mc, part, counter, scal, gate); break;
        case 2: launch_pdl(k_pool_rms<2>, grid, dim3(32, 2, 2), 0, s, r, flags, d, rc, mc, part, counter, scal, gate); break;
        case 4: launch_pdl(k_pool_rms<4>, grid, dim3(32, 4, 4), 0, s, r, flags, d, rc, mc, part, counter, scal, gate); break;
        default: launch_pdl(k_pool_rms<8>, grid, dim3(32, 8, 4), 0, s, r, flags, d, rc, mc, part, counter, scal, gate); break;
    }
}
void prolong_dense(const float* yc, const float* mask, float* out, int Xf, int Yf, int Zf, int st, cudaStream_t s) {
    k_prolong_dense<<<blocks_for((size_t)Xf * Yf * Zf), 256, 0, s>>>(yc, mask, out, Xf, Yf, Zf, st);
}
void prolong_flags(const float* yc, const uint8_t* flags, const Dom& d, int st, float* out, cudaStream_t s,
                   const int* gate) {
    const dim3 grid((d.nx + 31) / 32, (d.ny + 7) / 8, (d.nz + kProlongKC - 1) / kProlongKC), blk(32, 8);
    switch (st) {
        case 1: launch_pdl(k_prolong_flags<1>, grid, blk, 0, s, yc, flags, d, out, gate); break;
        case 2: launch_pdl(k_prolong_flags<2>, grid, blk, 0, s, yc, flags, d, out, gate); break;
        case 4: launch_pdl(k_prolong_flags<4>, grid, blk, 0, s, yc, flags, d, out, gate); break;
        default: launch_pdl(k_prolong_flags<8>, grid, blk, 0, s, yc, flags, d, out, gate); break;
    }
}
void mse(const float* y, const float* t, const float* mask, float* g, double* loss, size_t n, double inv_n,
         cudaStream_t s) {
    k_mse<<<blocks_for(n), 256, 0, s>>>(y, t, mask, g, loss, n, inv_n);
}
void adam(float* w, float* m, float* v, const float* g, __nv_bfloat16* wb, size_t n, float lr, float b1, float b2,
          float eps, float c1, float c2, cudaStream_t s) {
    k_adam<<<blocks_for(n), 256, 0, s>>>(w, m, v, g, wb, n, lr, b1, b2, eps, c1, c2);
}
void to_bf16(const float* a, __nv_bfloat16* b, size_t n, cudaStream_t s) {
    k_to_bf16<<<blocks_for(n), 256, 0, s>>>(a, b, n);
}

// ---------------------------------------------------------------------------
// persistent network correction (one cooperative launch)

__device__ __forceinline__ uint64_t nn_global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// sense-counting grid barrier with a bounded wait (1 s); returns false (and
// records a timeout) if the other CTAs did not arrive in time
__device__ bool grid_barrier(unsigned* count, unsigned* gen, Scalars* sc) {
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g0 = *(volatile unsigned*)gen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(count, 1u) == gridDim.x - 1) {
            *(volatile unsigned*)count = 0u;
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const uint64_t t0 = nn_global_ns();
            while (*(volatile unsigned*)gen == g0)
                if (nn_global_ns() - t0 > 1000000000ull) {
                    ok = 0;
                    atomicExch(&sc->timeout, 1);
                    break;
                }
        }
        __threadfence();
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}

// block sum of NV doubles (fixed order), result on thread 0
template <int NV>
__device__ __forceinline__ void nn_block_sum(double (&x)[NV]) {
    __shared__ double sh[NV][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q)
        for (int o = 16; o > 0; o >>= 1) x[q] += __shfl_down_sync(0xffffffffu, x[q], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) sh[q][warp] = x[q];
    __syncthreads();
    if (warp == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            x[q] = lane < nw ? sh[q][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) x[q] += __shfl_down_sync(0xffffffffu, x[q], o);
        }
}

template <int IN>
__device__ void conv_phase(const ConvArgs& A, ConvStage<16>* st) {
    const int ntx = (A.X + TX - 1) / TX, nty = (A.Y + TY - 1) / TY, ntz = (A.Z + TZ - 1) / TZ;
    const int tiles = ntx * nty * ntz * (A.Cout / 16);
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
        conv_tile<16, IN>(A, t % ntx, (t / ntx) % nty, t / (ntx * nty), st);
        __syncthreads();
    }
}

// the coarse network in one launch: RMS of the pooled residual, packing, the
// seven convolutions (pooling / upsampling folded into their staging) and the
// head, phases separated by the grid barrier.  The pooled residual and mask
// come from the pooling kernel; prolongation, line search and step follow as
// ordinary full-grid kernels.
__global__ void __launch_bounds__(256) k_net_infer(const __grid_constant__ NetInferArgs A) {
    extern __shared__ __align__(16) unsigned char infer_smem[];
    ConvStage<16>* st = reinterpret_cast<ConvStage<16>*>(infer_smem);
    Scalars* sc = A.sc;
    if (A.gate && *(volatile const int*)A.gate) return;      // uniform: the solve has ended
    const int Xc = A.L[0][0], Yc = A.L[0][1], Zc = A.L[0][2];
    const int nc = Xc * Yc * Zc;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
    // 1. RMS partials per CTA: sum mask r^2 and sum mask
    double rs[2] = {0.0, 0.0};
    for (int c = gt; c < nc; c += gs) {
        const double rv = A.rc[c], mv = A.mask[c];
        rs[0] += mv * rv * rv;
        rs[1] += mv;
    }
    nn_block_sum<2>(rs);
    if (threadIdx.x == 0) {
        A.cta[2 * blockIdx.x] = rs[0];
        A.cta[2 * blockIdx.x + 1] = rs[1];
    }
    if (!grid_barrier(A.bar_count, A.bar_gen, sc)) return;
    // 2. RMS (every CTA adds the CTA partials in the same order) and the packed input
    double ts = 0.0, tm = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) {
        ts += A.cta[2 * b];
        tm += A.cta[2 * b + 1];
    }
    const double rms = tm > 0.0 ? sqrt(ts / tm) : 0.0;
    const float scale = (float)(rms > 0.0 ? 1.0 / rms : 0.0);
    for (int c = gt; c < nc; c += gs) {
        __align__(16) __nv_bfloat16 o[16];
        o[0] = __float2bfloat16(A.mask[c] * A.rc[c] * scale);
        o[1] = __float2bfloat16(A.mask[c]);
#pragma unroll
        for (int ch = 2; ch < 16; ++ch) o[ch] = __float2bfloat16(0.f);
        uint4* dst = reinterpret_cast<uint4*>(A.xin + (size_t)c * 16);
        dst[0] = reinterpret_cast<const uint4*>(o)[0];
        dst[1] = reinterpret_cast<const uint4*>(o)[1];
    }
    if (!grid_barrier(A.bar_count, A.bar_gen, sc)) return;
    // 3. the U-Net
    const int(*L)[3] = A.L;
    {
        const ConvArgs c0{A.xin, A.wb[0], A.e[0], nullptr, nullptr, L[0][0], L[0][1], L[0][2], 16, 16, 1,
                          L[0][0], L[0][1], L[0][2]};
        conv_phase<IN_DIRECT>(c0, st);
    }
    if (!grid_barrier(A.bar_count, A.bar_gen, sc)) return;
    {
        const ConvArgs c1{A.e[0], A.wb[1], A.e[1], nullptr, nullptr, L[1][0], L[1][1], L[1][2], 16, 32, 1,
                          L[0][0], L[0][1], L[0][2]};
        conv_phase<IN_POOL>(c1, st);
    }
    if (!grid_barrier(A.bar_count, A.bar_gen, sc)) return;
    {
        const ConvArgs c2{A.e[1], A.wb[2], A.e[2], nullptr, nullptr, L[2][0], L[2][1], L[2][2], 32, 64, 1,
                          L[1][0], L[1][1], L[1][2]};
        conv_phase<IN_POOL>(c2, st);
    }
    if (!grid_barrier(A.bar_count, A.bar_gen, sc)) return;
    {
        const ConvArgs c3{A.e[2], A.wb[3], A.e[3], nullptr, nullptr, L[3][0], L[3][1], L[3][2], 64, 128, 1,
                          L[2][0], L[2][1], L[2][2]};
        conv_phase<IN_POOL>(c3, st);
    }
    if (!grid_barrier(A.bar_count, A.bar_gen, sc)) return;
    {
        const ConvArgs c4{A.e[3], A.wb[4], A.rr[2], A.e[2], A.dd[2], L[2][0], L[2][1], L[2][2], 128, 64, 1,
                          L[3][0], L[3][1], L[3][2]};
        conv_phase<IN_UP>(c4, st);
    }
    if (!grid_barrier(A.bar_count, A.bar_gen, sc)) return;
    {
        const ConvArgs c5{A.dd[2], A.wb[5], A.rr[1], A.e[1], A.dd[1], L[1][0], L[1][1], L[1][2], 64, 32, 1,
                          L[2][0], L[2][1], L[2][2]};
        conv_phase<IN_UP>(c5, st);
    }
    if (!grid_barrier(A.bar_count, A.bar_gen, sc)) return;
    {
        const ConvArgs c6{A.dd[1], A.wb[6], A.rr[0], A.e[0], A.dd[0], L[0][0], L[0][1], L[0][2], 32, 16, 1,
                          L[1][0], L[1][1], L[1][2]};
        conv_phase<IN_UP>(c6, st);
    }
    if (!grid_barrier(A.bar_count, A.bar_gen, sc)) return;
    // 4. head
    for (int c = gt; c < nc; c += gs) {
        float sacc = 0.f;
        for (int ch = 0; ch < 16; ++ch) sacc += A.head_w[ch] * __bfloat162float(A.dd[0][(size_t)c * 16 + ch]);
        A.y[c] = A.mask[c] * sacc;
    }
}

int net_infer_grid() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 0;
    if (cached[dev]) return cached[dev] > 0 ? cached[dev] : 0;
    int coop = 0, sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int smem = (int)(2 * sizeof(ConvStage<16>));
    if (cudaFuncSetAttribute(k_net_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_net_infer, 256, smem) != cudaSuccess || !coop ||
        per_sm < 1) {
        cudaGetLastError();
        cached[dev] = -1;
        return 0;
    }
    cached[dev] = sms;          // one CTA per SM: cheap barriers, enough for the coarse grid
    return sms;
}

cudaError_t net_infer_launch(const NetInferArgs& a, int grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 2 * sizeof(ConvStage<16>);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaMemsetAsync(a.bar_count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, k_net_infer, a);
}

}  // namespace nn
}  // namespace les
