// pt_surrogate.cu -- BF16 tensor-core inference of the surrogate network for
// the ingress/egress Mandel-Agol terms, with the exact kernel as fallback
// (the network is not in the paper; its analogue there is the
// interpolation tables of Sec. 2.2.3).
//
// One persistent CTA of 128 threads per tile of 128 points (several tiles
// per CTA):
//   layer 1 (2 -> 128) on the CUDA cores, one point per thread, BF16 result
//     written to shared memory in the tensor cores' K-major layout;
//   layers 2 and 3 (128 x 128) as tcgen05.mma kind::f16 (BF16 x BF16 -> FP32)
//     with A (activations) and B (weights) in shared memory and the
//     accumulator in tensor memory; one thread issues 8 MMAs (K = 16 each)
//     and tcgen05.commit arrives on an mbarrier when they finish;
//   epilogues read the accumulator with tcgen05.ld (warp w owns TMEM lanes
//     32w..32w+31 = rows of the tile), add the bias, apply SiLU, and store
//     BF16 for the next MMA (layer 2) or keep FP32 for layer 4 (128 -> 2,
//     CUDA cores);
//   de-normalisation, and the exact kernel for points outside the band or
//     in a cell the error-bound table marks.
// Every mbarrier wait is bounded; on time-out the kernel records an error,
// stops issuing work, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "../../include/pt.h"
#include "pt_device.cuh"

namespace pt_internal {
int set_error(int status, const char *where, const char *msg);   // pt_lc.cu
}

namespace {

constexpr int H = PT_MLP_HIDDEN;
constexpr int TILE = 128;                 // points per tile = MMA M
constexpr int NTHR = 256;                 // 8 warps
constexpr int TILE_BYTES = H * H * 2;     // one 128 x 128 BF16 operand (32 KB)
constexpr int TMEM_COLS = 128;            // FP32 accumulator 128 x 128
constexpr long long WAIT_LIMIT = 1 << 22; // bounded mbarrier polls

constexpr int OFF_W1 = 0, OFF_B1 = 2 * H, OFF_W2 = 3 * H, OFF_B2 = 3 * H + H * H, OFF_W3 = 4 * H + H * H,
              OFF_B3 = 4 * H + 2 * H * H, OFF_W4 = 5 * H + 2 * H * H, OFF_B4 = 7 * H + 2 * H * H;

int cuda_status(const char *where)
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PT_OK : pt_internal::set_error(PT_ERR_CUDA, where, cudaGetErrorString(e));
}

// K-major operand layout without swizzle, built from 8 x 8 "core matrices"
// (8 rows of 16 contiguous bytes = 128 B): element (row r, column k) sits at
//   (r / 8) * SBO + (k / 8) * LBO + (r % 8) * 16 + (k % 8) * 2,
// with LBO = 128 B between core matrices adjacent along K and
// SBO = (H / 8) * 128 B = 2048 B between 8-row groups.
constexpr uint32_t LBO = 128, SBO = (H / 8) * 128;

__host__ __device__ __forceinline__ uint32_t op_offset(int r, int k)
{
    return (uint32_t)(r >> 3) * SBO + (uint32_t)(k >> 3) * LBO + (uint32_t)(r & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

// tcgen05 shared-memory matrix descriptor: start address >> 4 (bits 0-13),
// LBO >> 4 (16-29), SBO >> 4 (32-45), the fixed 0b001 of bits 46-48, no
// swizzle (bits 61-63 = 0), base offset 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(LBO >> 4) << 16;
    d |= (uint64_t)(SBO >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(H >> 3) << 17) |
                           ((uint32_t)(TILE >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Bounded wait for the mbarrier phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t addr = smem_u32(bar);
    for (long long it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] x B[smem]^T over K = 128: 8 MMAs of K = 16, then commit.
__device__ __forceinline__ void issue_layer(uint32_t tmem_d, uint32_t a_base, uint32_t b_base, uint64_t *bar)
{
#pragma unroll
    for (int kk = 0; kk < H / 16; ++kk) {
        uint64_t ad = smem_desc(a_base + (uint32_t)kk * 2u * LBO);
        uint64_t bd = smem_desc(b_base + (uint32_t)kk * 2u * LBO);
        uint32_t acc = kk > 0 ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(tmem_d), "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
            : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive FP32 accumulator columns of this thread's row.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// SiLU through tanh: x sigma(x) = x (1 + tanh(x/2)) / 2 (one MUFU op).  Its
// ~2^-11 relative error is below the BF16 rounding that follows it.
__device__ __forceinline__ float silu_fast(float x)
{
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * x));
    return 0.5f * x * (1.0f + t);
}

__device__ __forceinline__ float silu_acc(float x) { return x / (1.0f + expf(-x)); }

struct SurModel {
    const float *p32;          // FP32 parameters (W1, b1, b2, b3, W4, b4 used from here)
    const __nv_bfloat16 *w2;   // W2 in the operand layout
    const __nv_bfloat16 *w3;   // W3 in the operand layout
    float norm[6];
    float k_lo, k_hi;
    const unsigned char *table;   // [nk][ns], 1 = exact
    int nk, ns;
};

struct SurArgs {
    SurModel m;
    int mode;                  // 0: network outputs Y from X; 1: surrogate MA terms for listed points
    const float *X;            // mode 0: [n][2]
    float *Y;                  // mode 0: [n][2]
    const float *k, *z;        // mode 1
    float *le, *ld, *ed;       // mode 1
    const int *list;           // mode 1: indices of the points the network serves
    const int *count;          // mode 1: number of listed points (device)
    size_t n;                  // mode 0: number of points
    int *err;                  // set to 1 on an mbarrier time-out
};

// Classify every point: outside the band or in a marked cell -> exact
// kernel here and now; otherwise append to the network's list.
__global__ void classify_kernel(SurModel m, const float *k, const float *z, size_t n, float *le, float *ld,
                                float *ed, int *list, int *count, int *n_fallback)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool net = false;
    if (i < n) {
        float kk = k[i], zz = fabsf(z[i]);
        float s = (zz - fabsf(1.0f - kk)) / (2.0f * fminf(kk, 1.0f));
        net = kk >= m.k_lo && kk <= m.k_hi && s >= 0.0f && s < 1.0f;
        if (net) {
            int ck = min(m.nk - 1, (int)((kk - m.k_lo) / (m.k_hi - m.k_lo) * m.nk));
            int cs = min(m.ns - 1, (int)(s * m.ns));
            net = m.table[ck * m.ns + cs] == 0;
        }
        if (!net) {
            float a, b, c;
            pt::ma_terms(kk, zz, &a, &b, &c);
            le[i] = a;
            ld[i] = b;
            ed[i] = c;
        }
    }
    // warp-aggregated appends
    unsigned mask = __ballot_sync(0xffffffffu, net);
    int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0 && mask) base = atomicAdd(count, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (net) list[base + __popc(mask & ((1u << lane) - 1u))] = (int)i;
    unsigned fb = __ballot_sync(0xffffffffu, i < n && !net);
    if (lane == 0 && fb && n_fallback) atomicAdd(n_fallback, __popc(fb));
}

// Thread layout: 8 warps; warp w serves tile rows 32 (w % 4) .. +31 (the
// tensor-memory lanes it may read) and columns 64 (w / 4) .. +63.
__global__ void __launch_bounds__(NTHR) sur_kernel(SurArgs A)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem;                        // activations, 32 KB
    unsigned char *sW2 = smem + TILE_BYTES;          // 32 KB
    unsigned char *sW3 = smem + 2 * TILE_BYTES;      // 32 KB
    float *sW1 = reinterpret_cast<float *>(smem + 3 * TILE_BYTES);   // [128][2]
    float *sB1 = sW1 + 2 * H;
    float *sB2 = sB1 + H;
    float *sB3 = sB2 + H;
    float *sW4 = sB3 + H;                                           // [2][128]
    float *sY = sW4 + 2 * H;                                        // [128][2] partial outputs
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = 32 * (warp & 3) + (tid & 31);
    const int half = warp >> 2, c0 = 64 * half;
    {
        const uint4 *g2 = reinterpret_cast<const uint4 *>(A.m.w2);
        const uint4 *g3 = reinterpret_cast<const uint4 *>(A.m.w3);
        uint4 *d2 = reinterpret_cast<uint4 *>(sW2);
        uint4 *d3 = reinterpret_cast<uint4 *>(sW3);
        for (int i = tid; i < TILE_BYTES / 16; i += NTHR) {
            d2[i] = g2[i];
            d3[i] = g3[i];
        }
        for (int i = tid; i < 2 * H; i += NTHR) {
            sW1[i] = A.m.p32[OFF_W1 + i];
            sW4[i] = A.m.p32[OFF_W4 + i];
        }
        for (int i = tid; i < H; i += NTHR) {
            sB1[i] = A.m.p32[OFF_B1 + i];
            sB2[i] = A.m.p32[OFF_B2 + i];
            sB3[i] = A.m.p32[OFF_B3 + i];
        }
    }
    if (tid == 0) {
        mbar_init(&bar, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"((uint32_t)TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t aA = smem_u32(sA), aW2 = smem_u32(sW2), aW3 = smem_u32(sW3);
    const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0;
    const float b4_0 = A.m.p32[OFF_B4], b4_1 = A.m.p32[OFF_B4 + 1];
    const size_t n = (A.mode == 0) ? A.n : (size_t)(*A.count);
    const size_t n_tiles = (n + TILE - 1) / TILE;
    uint32_t phase = 0;   // parity of the next mbarrier phase to complete

    for (size_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const size_t slot = tile * TILE + row;
        const bool valid = slot < n;
        size_t i = slot;
        float x0 = 0.0f, x1 = 0.0f, kk = 0.1f, zz = 1.0f;
        if (valid) {
            if (A.mode == 0) {
                x0 = A.X[2 * i];
                x1 = A.X[2 * i + 1];
            } else {
                i = (size_t)A.list[slot];
                kk = A.k[i];
                zz = fabsf(A.z[i]);
                float s = (zz - fabsf(1.0f - kk)) / (2.0f * fminf(kk, 1.0f));
                x0 = (kk - A.m.norm[0]) / A.m.norm[1];
                x1 = pt::band_coord(fminf(1.0f, fmaxf(0.0f, s)));
            }
        }
        // ---- layer 1 (this thread's 64 columns) -> BF16 operand
#pragma unroll 2
        for (int k0 = c0; k0 < c0 + 64; k0 += 8) {
            __align__(16) __nv_bfloat16 h8[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                int j = k0 + q;
                float zj = fmaf(sW1[2 * j], x0, fmaf(sW1[2 * j + 1], x1, sB1[j]));
                h8[q] = __float2bfloat16_rn(silu_fast(zj));
            }
            *reinterpret_cast<uint4 *>(sA + op_offset(row, k0)) = *reinterpret_cast<uint4 *>(h8);
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0 && !s_abort) issue_layer(tmem, aA, aW2, &bar);
        bool ok = mbar_wait(&bar, phase);
        phase ^= 1u;
        if (!ok) s_abort = 1;
        tc_fence_after();
        __syncthreads();
        if (s_abort) break;
        // ---- epilogue 2
#pragma unroll 1
        for (int c = 0; c < 64; c += 32) {
            float v[32];
            tmem_ld32(trow + (uint32_t)c, v);
#pragma unroll
            for (int k0 = 0; k0 < 32; k0 += 8) {
                __align__(16) __nv_bfloat16 h8[8];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    h8[q] = __float2bfloat16_rn(silu_fast(v[k0 + q] + sB2[c0 + c + k0 + q]));
                *reinterpret_cast<uint4 *>(sA + op_offset(row, c0 + c + k0)) = *reinterpret_cast<uint4 *>(h8);
            }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0 && !s_abort) issue_layer(tmem, aA, aW3, &bar);
        ok = mbar_wait(&bar, phase);
        phase ^= 1u;
        if (!ok) s_abort = 1;
        tc_fence_after();
        __syncthreads();
        if (s_abort) break;
        // ---- epilogue 3 + layer 4 partial sums over this thread's columns
        float y0 = 0.0f, y1 = 0.0f;
#pragma unroll 1
        for (int c = 0; c < 64; c += 32) {
            float v[32];
            tmem_ld32(trow + (uint32_t)c, v);
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                int j = c0 + c + q;
                float h = silu_acc(v[q] + sB3[j]);
                y0 = fmaf(sW4[j], h, y0);
                y1 = fmaf(sW4[H + j], h, y1);
            }
        }
        if (half == 1) {
            sY[2 * row] = y0;
            sY[2 * row + 1] = y1;
        }
        tc_fence_before();
        __syncthreads();   // partial sums exchanged; accumulator fully read before the next MMA
        tc_fence_after();
        if (half == 0 && valid) {
            y0 += sY[2 * row] + b4_0;
            y1 += sY[2 * row + 1] + b4_1;
            if (A.mode == 0) {
                A.Y[2 * i] = y0;
                A.Y[2 * i + 1] = y1;
            } else {
                float k2 = kk * kk;
                A.le[i] = pt::lens_le(kk, zz);
                A.ld[i] = k2 * fmaf(y0, A.m.norm[3], A.m.norm[2]);
                A.ed[i] = k2 * fmaf(y1, A.m.norm[5], A.m.norm[4]);
            }
        }
    }
    if (s_abort) mbar_wait(&bar, phase ^ 1u);   // in-flight MMAs finish before the memory is freed
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0 && s_abort && A.err) atomicExch(A.err, 1);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)TMEM_COLS)
                     : "memory");
}

// Per-cell maximum of the flux-error bound 4 |d lambda_d| + 2 |d eta_d| of the
// network against the exact kernel over validation points (k, z) in the
// band; |weights| <= 4 and 2 bound the quadratic-law coefficients of
// lambda_d and eta_d in Eq. (ma_model) for q1, q2 in [0, 1].  Non-negative
// floats order like their bit patterns, so atomicMax on the bits is exact.
__global__ void cell_error_kernel(const float *k, const float *z, const float *ld_ref, const float *ed_ref,
                                  const float *ld_sur, const float *ed_sur, size_t n, float k_lo, float k_hi, int nk,
                                  int ns, unsigned int *cell_max)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float kk = k[i], zz = fabsf(z[i]);
    float s = (zz - fabsf(1.0f - kk)) / (2.0f * fminf(kk, 1.0f));
    if (!(kk >= k_lo && kk <= k_hi && s >= 0.0f && s < 1.0f)) return;
    int ck = min(nk - 1, (int)((kk - k_lo) / (k_hi - k_lo) * nk));
    int cs = min(ns - 1, (int)(s * ns));
    float e = 4.0f * fabsf(ld_sur[i] - ld_ref[i]) + 2.0f * fabsf(ed_sur[i] - ed_ref[i]);
    if (!(e >= 0.0f)) e = 3.0e38f;   // NaN counts as failure
    atomicMax(&cell_max[ck * ns + cs], __float_as_uint(e));
}

// W (FP32 [128 out][128 in], rows = N, K contiguous) -> BF16 operand layout.
__global__ void pack_weights_kernel(const float *W, __nv_bfloat16 *out)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= H * H) return;
    int r = idx / H, k = idx % H;
    out[op_offset(r, k) / 2] = __float2bfloat16_rn(W[idx]);
}

size_t sur_smem() { return (size_t)3 * TILE_BYTES + (size_t)(2 * H + 3 * H + 2 * H + 2 * TILE) * sizeof(float); }

}  // namespace

struct pt_sur_model_s {
    SurModel m;
    float *d_p32;
    __nv_bfloat16 *d_w2, *d_w3;
    unsigned char *d_table;
    int *d_err;
    int grid;
};

extern "C" {

int pt_sur_model_create(const float *params_dev, const float *norm, float k_lo, float k_hi,
                        const unsigned char *table, int nk, int ns, pt_sur_model *out)
{
    if (!params_dev || !norm || !table || !out || nk < 1 || ns < 1 || !(k_lo > 0.0f) || !(k_hi > k_lo) ||
        k_hi > 1.0f)
        return PT_ERR_ARG;
    *out = nullptr;
    pt_sur_model_s *p = new pt_sur_model_s();
    cudaError_t e = cudaMalloc(&p->d_p32, PT_MLP_NPARAMS * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_w2, TILE_BYTES);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_w3, TILE_BYTES);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_table, (size_t)nk * ns);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(p->d_p32, params_dev, PT_MLP_NPARAMS * sizeof(float), cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_table, table, (size_t)nk * ns, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int));
    if (e == cudaSuccess) {
        pack_weights_kernel<<<(H * H + 255) / 256, 256>>>(p->d_p32 + OFF_W2, p->d_w2);
        pack_weights_kernel<<<(H * H + 255) / 256, 256>>>(p->d_p32 + OFF_W3, p->d_w3);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sur_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sur_smem());
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sur_kernel, NTHR, sur_smem());
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || per_sm < 1) {
        int st = pt_internal::set_error(PT_ERR_CUDA, "pt_sur_model_create",
                                        e != cudaSuccess ? cudaGetErrorString(e) : "no resident CTA fits");
        cudaFree(p->d_p32);
        cudaFree(p->d_w2);
        cudaFree(p->d_w3);
        cudaFree(p->d_table);
        cudaFree(p->d_err);
        delete p;
        return st;
    }
    p->grid = nsm * per_sm;
    p->m.p32 = p->d_p32;
    p->m.w2 = p->d_w2;
    p->m.w3 = p->d_w3;
    for (int i = 0; i < 6; ++i) p->m.norm[i] = norm[i];
    p->m.k_lo = k_lo;
    p->m.k_hi = k_hi;
    p->m.table = p->d_table;
    p->m.nk = nk;
    p->m.ns = ns;
    *out = p;
    return PT_OK;
}

int pt_sur_model_destroy(pt_sur_model p)
{
    if (!p) return PT_OK;
    cudaFree(p->d_p32);
    cudaFree(p->d_w2);
    cudaFree(p->d_w3);
    cudaFree(p->d_table);
    cudaFree(p->d_err);
    delete p;
    return PT_OK;
}

static int launch_sur(pt_sur_model p, SurArgs &a, size_t max_points, pt_stream_t stream)
{
    a.m = p->m;
    a.err = p->d_err;
    size_t tiles = (max_points + TILE - 1) / TILE;
    int grid = (int)(tiles < (size_t)p->grid ? tiles : (size_t)p->grid);
    if (grid < 1) grid = 1;
    sur_kernel<<<grid, NTHR, sur_smem(), (cudaStream_t)stream>>>(a);
    return cuda_status("sur_kernel");
}

int pt_sur_mlp_eval(pt_sur_model p, const float *X, size_t n, float *Y, pt_stream_t stream)
{
    if (!p) return PT_ERR_ARG;
    if (n == 0) return PT_OK;
    if (!X || !Y) return PT_ERR_ARG;
    SurArgs a{};
    a.mode = 0;
    a.X = X;
    a.Y = Y;
    a.n = n;
    return launch_sur(p, a, n, stream);
}

size_t pt_sur_work_bytes(size_t n) { return 256 + ((n * sizeof(int) + 255) & ~(size_t)255); }

int pt_ma_surrogate(pt_sur_model p, const float *k, const float *z, size_t n, float *le, float *ld, float *ed,
                    int *n_fallback, void *work, size_t work_bytes, pt_stream_t stream)
{
    if (!p) return PT_ERR_ARG;
    if (n == 0) return PT_OK;
    if (!k || !z || !le || !ld || !ed) return PT_ERR_ARG;
    if (n > 0x7fffffffULL) return PT_ERR_ARG;
    if (!work || work_bytes < pt_sur_work_bytes(n)) return PT_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    int *count = (int *)work;
    int *list = (int *)((char *)work + 256);
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), s);
    if (e != cudaSuccess) return pt_internal::set_error(PT_ERR_CUDA, "pt_ma_surrogate", cudaGetErrorString(e));
    size_t blocks = (n + 255) / 256;
    classify_kernel<<<(unsigned)blocks, 256, 0, s>>>(p->m, k, z, n, le, ld, ed, list, count, n_fallback);
    int st = cuda_status("classify_kernel");
    if (st) return st;
    SurArgs a{};
    a.mode = 1;
    a.k = k;
    a.z = z;
    a.le = le;
    a.ld = ld;
    a.ed = ed;
    a.list = list;
    a.count = count;
    return launch_sur(p, a, n, stream);
}

int pt_sur_model_error(pt_sur_model p, int *err_host)
{
    if (!p || !err_host) return PT_ERR_ARG;
    cudaError_t e = cudaMemcpy(err_host, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? PT_OK : pt_internal::set_error(PT_ERR_CUDA, "pt_sur_model_error", cudaGetErrorString(e));
}

int pt_sur_cell_errors(const float *k, const float *z, const float *ld_ref, const float *ed_ref, const float *ld_sur,
                       const float *ed_sur, size_t n, float k_lo, float k_hi, int nk, int ns, float *cell_max,
                       pt_stream_t stream)
{
    if (n == 0) return PT_OK;
    if (!k || !z || !ld_ref || !ed_ref || !ld_sur || !ed_sur || !cell_max || nk < 1 || ns < 1) return PT_ERR_ARG;
    size_t blocks = (n + 255) / 256;
    if (blocks > 0x7fffffffULL) return PT_ERR_ARG;
    cell_error_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(k, z, ld_ref, ed_ref, ld_sur, ed_sur, n,
                                                                          k_lo, k_hi, nk, ns,
                                                                          reinterpret_cast<unsigned int *>(cell_max));
    return cuda_status("cell_error_kernel");
}

}  // extern "C"
