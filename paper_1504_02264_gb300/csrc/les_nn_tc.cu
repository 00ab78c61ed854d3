// 3x3x3 convolution of the warm-start network on the fifth-generation tensor
// cores: implicit GEMM with tcgen05.mma (kind::f16, BF16 operands, FP32
// accumulator in tensor memory), issued by one thread per CTA.
//
// GEMM view: D[m][n] = sum_k A[m][k] B[n][k], m = one of the 128 output
// voxels of the CTA's tile (8 along x, 16 along y, one plane), n = output
// channel (CO = 16 or 32 per CTA), k = (tap, input channel).  Per 16-channel
// input chunk the CTA stages in shared memory
//   * the input halo block (10 x 18 x 3 voxels) as two 8-channel halves,
//     each half stored voxel after voxel at 16 bytes per voxel, so that the
//     8 x-consecutive voxels of a tile row, shifted by any tap, are eight
//     consecutive 16-byte rows: one 8x8 core matrix of the MMA's no-swizzle
//     K-major operand layout; the 16 tile rows are 160 bytes apart (the
//     stride between core matrices along M) and the two channel halves one
//     half-block apart (the stride along K).  One matrix descriptor per tap
//     therefore addresses the tap-shifted A operand without any copy;
//   * the chunk's weights [tap][half][co][8 ci] in the same layout (core
//     matrices 128 bytes apart along N, a half apart along K).
// Each chunk is 27 MMAs of 128 x CO x 16 (one per tap), accumulating in
// tensor memory.  Two stages: while the tensor cores work on one chunk the
// threads copy the next one in (cp.async); tcgen05.commit signals on an
// mbarrier when the MMAs reading a stage are done, before it is refilled.
// The epilogue reads the accumulator rows back with tcgen05.ld (warp w and
// w + 4 read lanes 32 (w % 4) .. + 31, each half of the columns), applies
// ReLU, rounds to BF16, adds the skip tensor, and stores NDHWC; small grids
// split the input-channel chunks over CTAs exactly as the warp-level kernel
// does (FP32 partials added in a fixed order by each tile's last CTA).
//
// Input staging modes match the warp-level kernel (direct, nearest
// upsampling of a coarser tensor, 2x2x2 mean pooling of a finer tensor with
// the same summation order), so both compute the same BF16 staged values.
// Every wait is bounded by the global timer; on a timeout the CTA records it,
// waits (bounded) for its MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "les_nn.cuh"

namespace les {
namespace nn {
namespace {

constexpr int TCX = 8, TCY = 16, HX = TCX + 2, HY = TCY + 2, HZ = 3;
constexpr int NVOX = HX * HY * HZ;                 // halo voxels per channel half
constexpr uint32_t HALF_A = NVOX * 16;             // bytes of one 8-channel half of the halo block
constexpr int NTH = 256;
constexpr size_t kTcSmemFloor = 0;

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void cp16(uint32_t dst, const void* src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N));
}

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait on one phase of an mbarrier (1 s of global time)
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = gtimer();
    while (!bar_try(bar, parity))
        if (gtimer() - t0 > 1000000000ull) return false;
    return true;
}

// shared-memory matrix descriptor, no swizzle, K-major: start address, the
// byte offset between core matrices along K (leading) and along M / N (stride)
__device__ __forceinline__ uint64_t mdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;                        // descriptor version of this architecture
    return d;                                      // base offset 0, layout type 0 (no swizzle)
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t dtm, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtm),
        "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
// thread-block cluster: barrier over every thread of every CTA (release /
// acquire), the address of the same shared variable in CTA `rank`, a 16-byte
// load from distributed shared memory
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_map(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ float4 cluster_ld4(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}

__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 8 (or 16) consecutive FP32 columns of this thread's accumulator row
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = __uint_as_float(r[c]);
}

template <int CO>
struct TcStage {
    __nv_bfloat16 a[2][NVOX][8];                  // [half][voxel (hz, hy, hx)][8 channels]
    __nv_bfloat16 b[27][2][CO][8];                // [tap][half][co][8 channels]
};

template <int CO>
struct TcSmem {
    TcStage<CO> st[2];
    uint64_t mma_done[2];
    uint32_t tmem;
};

// the input value of halo voxel (gx, gy, gz) of the output grid, 8 channels
// from c0: direct, nearest upsampling of a coarser tensor, or 2x2x2 mean
// pooling of a finer tensor (children outside the grid count as zero, summed
// in the order of the stand-alone pooling kernel)
template <int IN>
__device__ __forceinline__ void stage_half(const ConvArgs& A, int gx, int gy, int gz, int c0, uint32_t dst,
                                           __nv_bfloat16* dstp) {
    const bool ok = gx >= 0 && gx < A.X && gy >= 0 && gy < A.Y && gz >= 0 && gz < A.Z;
    if constexpr (IN == IN_POOL) {
        float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (ok) {
            uint4 ch[8];
            bool in[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int fx = 2 * gx + (e & 1), fy = 2 * gy + ((e >> 1) & 1), fz = 2 * gz + (e >> 2);
                in[e] = fx < A.Xs && fy < A.Ys && fz < A.Zs;
                ch[e] = in[e] ? *reinterpret_cast<const uint4*>(A.x + (((size_t)fz * A.Ys + fy) * A.Xs + fx) * A.Cin + c0)
                              : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (in[e]) {
                    const __nv_bfloat16* b = reinterpret_cast<const __nv_bfloat16*>(&ch[e]);
#pragma unroll
                    for (int c = 0; c < 8; ++c) a[c] += __bfloat162float(b[c]);
                }
        }
        __align__(16) __nv_bfloat16 o[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) o[c] = __float2bfloat16(0.125f * a[c]);
        *reinterpret_cast<uint4*>(dstp) = *reinterpret_cast<const uint4*>(o);
    } else if constexpr (IN == IN_PACK) {
        __align__(16) __nv_bfloat16 o[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) o[c] = __float2bfloat16(0.f);
        if (ok && c0 == 0) {
            const size_t v = ((size_t)gz * A.Y + gy) * A.X + gx;
            const double sc = A.pscale[0];
            const float s = (float)(sc > 0.0 ? 1.0 / sc : 0.0);
            o[0] = __float2bfloat16(A.pmask[v] * A.prc[v] * s);
            o[1] = __float2bfloat16(A.pmask[v]);
        }
        *reinterpret_cast<uint4*>(dstp) = *reinterpret_cast<const uint4*>(o);
    } else {
        const int sx = IN == IN_UP ? gx >> 1 : gx, sy = IN == IN_UP ? gy >> 1 : gy, sz = IN == IN_UP ? gz >> 1 : gz;
        const __nv_bfloat16* src = ok ? A.x + (((size_t)sz * A.Ys + sy) * A.Xs + sx) * A.Cin + c0 : A.x;
        cp16(dst, src, ok ? 16 : 0);
    }
}

template <int CO, int IN>
__global__ void __launch_bounds__(NTH) k_conv3_tc(ConvArgs A, const int* gate, int* timeout) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    TcSmem<CO>& S = *reinterpret_cast<TcSmem<CO>*>(tc_smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int X = A.X, Y = A.Y, Z = A.Z, Cin = A.Cin, Cout = A.Cout;
    const int ks = A.ks > 1 ? A.ks : 1;
    const int kq = blockIdx.z % ks, bz = blockIdx.z / ks;
    const int x0 = blockIdx.x * TCX, y0 = blockIdx.y * TCY, z0 = bz % Z, co0 = (bz / Z) * CO;
    const int nch = Cin / 16, cb = kq * nch / ks, ce = (kq + 1) * nch / ks;
    constexpr uint32_t TM_COLS = 32;               // accumulator: 128 lanes x CO <= 32 FP32 columns
    constexpr uint32_t ID = idesc_bf16(128, CO);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&S.tmem)),
                     "r"(TM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        bar_init(saddr(&S.mma_done[0]), 1);
        bar_init(saddr(&S.mma_done[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = S.tmem;

    // a chunk's weights (no kernel of the solve writes them) and its input halo
    auto stage_w = [&](int c, TcStage<CO>& T) {
        const int c0 = 16 * c;
        for (int q = tid; q < 27 * 2 * CO; q += NTH) {
            const int co = q % CO, h = (q / CO) & 1, tap = q / (2 * CO);
            const bool ok = co0 + co < Cout;
            const __nv_bfloat16* src = ok ? A.w + ((size_t)tap * Cout + co0 + co) * Cin + c0 + 8 * h : A.w;
            cp16(saddr(&T.b[tap][h][co][0]), src, ok ? 16 : 0);
        }
    };
    auto stage_x = [&](int c, TcStage<CO>& T) {
        const int c0 = 16 * c;
        for (int q = tid; q < 2 * NVOX; q += NTH) {
            const int h = q / NVOX, v = q % NVOX;
            const int hx = v % HX, hy = (v / HX) % HY, hz = v / (HX * HY);
            stage_half<IN>(A, x0 - 1 + hx, y0 - 1 + hy, z0 - 1 + hz, c0 + 8 * h, saddr(&T.a[h][v][0]), &T.a[h][v][0]);
        }
    };
    auto stage = [&](int c, TcStage<CO>& T) {
        stage_x(c, T);
        stage_w(c, T);
        cp_commit();
    };

    bool ok = true;
    int issued = cb - 1;                           // the last chunk whose MMAs were issued
    // The packed, pooled and upsampled layers run only inside an inference of
    // the solve, right after the pooling kernel or the previous convolution,
    // neither of which writes weights (and every kernel before those has
    // completed by the time this one can launch): their first chunk's weights
    // are copied before the wait for that kernel (its tail overlaps the
    // copies).  Every layer lets the next kernel launch once the wait has
    // returned (every kernel that follows a convolution waits for it before it
    // reads anything the convolution writes).
    constexpr bool kWeightsEarly = IN == IN_PACK || IN == IN_POOL || IN == IN_UP;
    if constexpr (kWeightsEarly) stage_w(cb, S.st[0]);
    pdl_wait();
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // the solve this inference serves may have ended: the flag's load is
    // issued here and tested after the first chunk's copies are under way
    const int ended = gate ? *(volatile const int*)gate : 0;
    if constexpr (!kWeightsEarly) stage_w(cb, S.st[0]);
    stage_x(cb, S.st[0]);
    cp_commit();
    if (ended) {
        // uniform over the CTA: let the copies land, give the memory back
        cp_wait<0>();
        tc_before();
        __syncthreads();
        if (warp == 0) {
            tc_after();
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TM_COLS) : "memory");
        }
        return;
    }
    for (int c = cb; c < ce; ++c) {
        const int s = (c - cb) & 1;
        cp_wait<0>();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // staged data -> the tensor cores' reads
        __syncthreads();
        if (tid == 0) {
            tc_after();
            const uint32_t a0 = saddr(&S.st[s].a[0][0][0]), b0 = saddr(&S.st[s].b[0][0][0][0]);
#pragma unroll 1
            for (int tap = 0; tap < 27; ++tap) {
                const int dx = tap % 3, dy = (tap / 3) % 3, dz = tap / 9;
                const uint64_t ad = mdesc(a0 + (uint32_t)(((dz * HY + dy) * HX + dx) * 16), HALF_A, HX * 16);
                const uint64_t bd = mdesc(b0 + (uint32_t)(tap * 2 * CO * 16), CO * 16, 128);
                umma(tmem, ad, bd, ID, (c > cb || tap > 0) ? 1u : 0u);
            }
            umma_commit(saddr(&S.mma_done[s]));
        }
        issued = c;
        if (c + 1 < ce) {
            // the other stage was read by the previous chunk's MMAs
            if (c > cb && !bar_wait(saddr(&S.mma_done[s ^ 1]), (uint32_t)(((c - 1 - cb) >> 1) & 1))) ok = false;
            if (!__syncthreads_and(ok)) break;
            stage(c + 1, S.st[s ^ 1]);
        }
    }
    // the last issued chunk's MMAs (and with them every earlier one) have completed
    if (ok && issued >= cb) ok = bar_wait(saddr(&S.mma_done[(issued - cb) & 1]), (uint32_t)(((issued - cb) >> 1) & 1));
    ok = __syncthreads_and(ok);
    if (!ok) {
        if (tid == 0 && timeout) atomicExch(timeout, 1);
        // bounded grace for MMAs still in flight before the memory goes back
        if (tid == 0 && issued >= cb)
            bar_wait(saddr(&S.mma_done[(issued - cb) & 1]), (uint32_t)(((issued - cb) >> 1) & 1));
    }
    tc_after();
    // accumulator row (lane) 32 (w % 4) + lane: voxel (x0 + row % 8, y0 + row / 8);
    // warps 0-3 read columns 0 .. CO/2 - 1, warps 4-7 the rest, 8 at a time
    constexpr int NC = CO / 2;
    const int row = 32 * (warp & 3) + lane, cbase = (warp >> 2) * NC;
    float acc[NC];
    if (ok) {
#pragma unroll
        for (int g = 0; g < NC / 8; ++g) {
            float v[8];
            tmem_ld8(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(cbase + 8 * g), v);
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[8 * g + c] = v[c];
        }
    }
    tc_before();
    __syncthreads();
    if (warp == 0) {
        tc_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TM_COLS) : "memory");
    }
    if (ks > 1 && A.cluster) {
        // the split's CTAs form one thread-block cluster (rank = kq): each
        // leaves its accumulators in its own idle stage buffer, and after a
        // cluster barrier rank 0 adds them over distributed shared memory in
        // the order kq = 0, 1, ... (the sums of the global-memory path) and
        // runs the epilogue; a second barrier keeps every buffer alive until
        // it has been read.  Every CTA of the cluster reaches both barriers
        // (a CTA whose wait timed out contributes zeros and has flagged it).
        float4* mine = reinterpret_cast<float4*>(&S.st[0]) + tid * (NC / 4);
#pragma unroll
        for (int n = 0; n < NC / 4; ++n)
            mine[n] = ok ? make_float4(acc[4 * n], acc[4 * n + 1], acc[4 * n + 2], acc[4 * n + 3])
                         : make_float4(0.f, 0.f, 0.f, 0.f);
        cluster_sync();
        if (kq == 0 && ok) {
#pragma unroll
            for (int n = 0; n < NC; ++n) acc[n] = 0.f;
            const uint32_t own = saddr(mine);
            for (int k = 0; k < ks; ++k) {
                const uint32_t peer = cluster_map(own, (uint32_t)k);
#pragma unroll
                for (int n = 0; n < NC / 4; ++n) {
                    const float4 v = cluster_ld4(peer + 16u * n);
                    acc[4 * n] += v.x;
                    acc[4 * n + 1] += v.y;
                    acc[4 * n + 2] += v.z;
                    acc[4 * n + 3] += v.w;
                }
            }
        }
        cluster_sync();
        if (kq != 0) return;
    }
    if (!ok) return;
    if (ks > 1 && !A.cluster) {
        // this split's accumulators; the tile's last CTA adds them in order
        __shared__ bool last;
        const size_t tile = (size_t)blockIdx.x + gridDim.x * ((size_t)blockIdx.y + gridDim.y * (size_t)bz);
        float4* mine = reinterpret_cast<float4*>(A.part) + ((tile * ks + kq) * NTH + tid) * (NC / 4);
#pragma unroll
        for (int n = 0; n < NC / 4; ++n) mine[n] = make_float4(acc[4 * n], acc[4 * n + 1], acc[4 * n + 2], acc[4 * n + 3]);
        __threadfence();
        __syncthreads();
        if (tid == 0) last = atomicAdd(&A.cnt[tile], 1u) == (unsigned)(ks - 1);
        __syncthreads();
        if (!last) return;
        __threadfence();
#pragma unroll
        for (int n = 0; n < NC; ++n) acc[n] = 0.f;
        for (int k = 0; k < ks; ++k) {
            const float4* p = reinterpret_cast<const float4*>(A.part) + ((tile * ks + k) * NTH + tid) * (NC / 4);
#pragma unroll
            for (int n = 0; n < NC / 4; ++n) {
                const float4 v = __ldcg(p + n);
                acc[4 * n] += v.x;
                acc[4 * n + 1] += v.y;
                acc[4 * n + 2] += v.z;
                acc[4 * n + 3] += v.w;
            }
        }
        if (tid == 0) A.cnt[tile] = 0u;
    }
    const int gx = x0 + (row & 7), gy = y0 + (row >> 3);
    if (A.head_y) {
        // the head: warps 0-3 sum channels 0-7 of their rows, warps 4-7 carry
        // the same rows' sums on through channels 8-15 (CO == Cout == 16)
        __shared__ float hsum[128];
        const bool valid = gx < X && gy < Y;
        const size_t o = (((size_t)z0 * Y + gy) * X + gx) * 16 + cbase;
        auto part = [&](float s) {
#pragma unroll
            for (int n = 0; n < NC; n += 2) {
                float v0 = acc[n], v1 = acc[n + 1];
                if (A.relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                const __nv_bfloat162 r = __floats2bfloat162_rn(v0, v1);
                const __nv_bfloat162 sk = *reinterpret_cast<const __nv_bfloat162*>(A.skip + o + n);
                const __nv_bfloat162 dv = __floats2bfloat162_rn(__bfloat162float(r.x) + __bfloat162float(sk.x),
                                                                __bfloat162float(r.y) + __bfloat162float(sk.y));
                s += A.head_w[cbase + n] * __bfloat162float(dv.x);
                s += A.head_w[cbase + n + 1] * __bfloat162float(dv.y);
            }
            return s;
        };
        if (warp < 4) hsum[row] = valid ? part(0.f) : 0.f;
        __syncthreads();
        if (warp >= 4 && valid) {
            const size_t v = ((size_t)z0 * Y + gy) * X + gx;
            A.head_y[v] = A.head_mask[v] * part(hsum[row]);
        }
        return;
    }
    if (gx >= X || gy >= Y) return;
    const size_t o = (((size_t)z0 * Y + gy) * X + gx) * Cout + co0 + cbase;
    if (co0 + cbase >= Cout) return;
#pragma unroll
    for (int n = 0; n < NC; n += 2) {
        float v0 = acc[n], v1 = acc[n + 1];
        if (A.relu) {
            v0 = fmaxf(v0, 0.f);
            v1 = fmaxf(v1, 0.f);
        }
        const __nv_bfloat162 r = __floats2bfloat162_rn(v0, v1);
        *reinterpret_cast<__nv_bfloat162*>(A.y + o + n) = r;
        if (A.skip) {
            const __nv_bfloat162 sk = *reinterpret_cast<const __nv_bfloat162*>(A.skip + o + n);
            *reinterpret_cast<__nv_bfloat162*>(A.ysum + o + n) =
                __floats2bfloat162_rn(__bfloat162float(r.x) + __bfloat162float(sk.x),
                                      __bfloat162float(r.y) + __bfloat162float(sk.y));
        }
    }
}

// dynamic shared memory per CTA: the two stages (kTcSmemFloor > 0 rounds the
// allocation up, so that any address a descriptor could form, with its
// strides read either way round, stays inside the CTA's shared memory)
template <int CO>
constexpr size_t tc_smem() {
    return sizeof(TcSmem<CO>) > kTcSmemFloor ? sizeof(TcSmem<CO>) : kTcSmemFloor;
}

template <int CO, int IN>
cudaError_t allow_tc() {
    return cudaFuncSetAttribute(k_conv3_tc<CO, IN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem<CO>());
}

// 1 when the current device co-schedules clusters of up to kMaxCluster CTAs
// of the largest convolution kernel (decided once per process, on the device
// current at the first preparation), else 0
constexpr int kMaxCluster = 8;
int g_tc_cluster = -1;

template <int CO, int IN>
cudaError_t tc_launch(dim3 grid, int cz, cudaStream_t s, const ConvArgs& A, const int* gate, int* timeout) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(NTH);
    cfg.dynamicSmemBytes = tc_smem<CO>();
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    int na = 1;
    if (cz > 1) {
        at[1].id = cudaLaunchAttributeClusterDimension;
        at[1].val.clusterDim.x = 1;
        at[1].val.clusterDim.y = 1;
        at[1].val.clusterDim.z = (unsigned)cz;
        na = 2;
    }
    cfg.attrs = at;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, k_conv3_tc<CO, IN>, A, gate, timeout);
}

}  // namespace

int conv3_tc_prepare() {
    cudaError_t e = cudaSuccess, x;
    if ((x = allow_tc<32, IN_DIRECT>()) != cudaSuccess) e = x;
    if ((x = allow_tc<16, IN_DIRECT>()) != cudaSuccess) e = x;
    if ((x = allow_tc<32, IN_UP>()) != cudaSuccess) e = x;
    if ((x = allow_tc<16, IN_UP>()) != cudaSuccess) e = x;
    if ((x = allow_tc<32, IN_POOL>()) != cudaSuccess) e = x;
    if ((x = allow_tc<16, IN_POOL>()) != cudaSuccess) e = x;
    if ((x = allow_tc<16, IN_PACK>()) != cudaSuccess) e = x;
    if (e == cudaSuccess && g_tc_cluster < 0) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(1, 1, kMaxCluster);
        cfg.blockDim = dim3(NTH);
        cfg.dynamicSmemBytes = tc_smem<32>();
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 1;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = kMaxCluster;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        const cudaError_t q = cudaOccupancyMaxActiveClusters(&n, k_conv3_tc<32, IN_UP>, &cfg);
        if (q != cudaSuccess) cudaGetLastError();
        g_tc_cluster = (q == cudaSuccess && n > 0) ? 1 : 0;
    }
    return e == cudaSuccess ? 0 : -1;
}

void conv3_tc_launch(ConvArgs A, int in_mode, cudaStream_t s, const int* gate, const ConvSplit* split, int* timeout,
                     bool cluster_split) {
    // 32 output channels per CTA when the grid fills the GPU, else 16; small
    // grids split their input-channel chunks over up to about two CTAs per SM
    const long long tiles = (long long)((A.X + TCX - 1) / TCX) * ((A.Y + TCY - 1) / TCY) * A.Z;
    const bool co16 = in_mode == IN_PACK || A.head_y;       // the modes built for 16 channels per CTA
    const int co = (!co16 && A.Cout >= 32 && tiles * (A.Cout / 32) >= 2 * 152) ? 32 : 16;
    dim3 grid((A.X + TCX - 1) / TCX, (A.Y + TCY - 1) / TCY, A.Z * ((A.Cout + co - 1) / co));
    int ks = 1;
    if (split) {
        const long long ctas = (long long)grid.x * grid.y * grid.z;
        const int nch = A.Cin / 16;
        while (nch % (2 * ks) == 0 && ctas * 2 * ks <= 2 * 152 &&
               (size_t)ctas * 2 * ks * NTH * (co / 2) <= split->part_floats && (size_t)ctas <= split->counters)
            ks *= 2;
        grid.z *= ks;
    }
    A.cluster = ks > 1 && ks <= kMaxCluster && cluster_split && g_tc_cluster == 1;
    A.part = ks > 1 && !A.cluster ? split->part : nullptr;
    A.cnt = ks > 1 && !A.cluster ? split->cnt : nullptr;
    A.ks = ks;
    const int cz = A.cluster ? ks : 1;
#define LES_TC_LAUNCH(CO_, IN_) tc_launch<CO_, IN_>(grid, cz, s, A, gate, timeout)
    if (in_mode == IN_PACK) {
        LES_TC_LAUNCH(16, IN_PACK);
    } else if (co == 32) {
        if (in_mode == IN_UP) LES_TC_LAUNCH(32, IN_UP);
        else if (in_mode == IN_POOL) LES_TC_LAUNCH(32, IN_POOL);
        else LES_TC_LAUNCH(32, IN_DIRECT);
    } else {
        if (in_mode == IN_UP) LES_TC_LAUNCH(16, IN_UP);
        else if (in_mode == IN_POOL) LES_TC_LAUNCH(16, IN_POOL);
        else LES_TC_LAUNCH(16, IN_DIRECT);
    }
#undef LES_TC_LAUNCH
}

}  // namespace nn
}  // namespace les
