// pt_mlp.cu -- training side of the surrogate network for the ingress/egress
// Mandel-Agol terms (the paper's analogue is the interpolation tables of
// Sec. 2.2.3; the network itself is not in the paper).
//
// Network: 2 -> 128 -> 128 -> 128 -> 2, SiLU, parameters flattened as
//   W1[128][2] b1[128] W2[128][128] b2[128] W3[128][128] b3[128] W4[2][128] b4[2].
// Loss: mean over samples of the summed squared output errors.
//
// Kernels: a counter-based (splitmix64) sampler of (k, s) whose targets come
// from the exact FP32 Mandel-Agol kernel; a tiled FP32 GEMM with fused
// epilogues (bias + SiLU, SiLU' product) whose operands can be rounded to
// BF16 (quantisation-aware fine-tuning, so the network is trained for the
// precision it is served in); deterministic split-K reductions for the
// weight gradients; Adam.
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
constexpr int NPAR = PT_MLP_NPARAMS;
constexpr int OFF_W1 = 0, OFF_B1 = 2 * H, OFF_W2 = 3 * H, OFF_B2 = 3 * H + H * H, OFF_W3 = 4 * H + H * H,
              OFF_B3 = 4 * H + 2 * H * H, OFF_W4 = 5 * H + 2 * H * H, OFF_B4 = 7 * H + 2 * H * H;
static_assert(OFF_B4 + 2 == NPAR, "parameter layout");
constexpr int SPLIT = 512;   // rows per split-K chunk of the weight gradients

int cuda_status(const char *where)
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PT_OK : pt_internal::set_error(PT_ERR_CUDA, where, cudaGetErrorString(e));
}

__device__ __forceinline__ float silu(float x) { return x / (1.0f + expf(-x)); }

__device__ __forceinline__ float dsilu(float x)
{
    float s = 1.0f / (1.0f + expf(-x));
    return s * (1.0f + x * (1.0f - s));
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// splitmix64 (Steele, Lea & Flood 2014): a counter-based 64-bit mixer
__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    x += 0x9e3779b97f4a7c15ULL;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
    return x ^ (x >> 31);
}

__device__ __forceinline__ float u01(uint64_t x)   // 24 random bits -> [0, 1)
{
    return (float)(x >> 40) * (1.0f / 16777216.0f);
}

__global__ void datagen_kernel(uint64_t seed, size_t offset, size_t n, float k_lo, float k_hi, const float *norm,
                               float *X, float *T, float *kz)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t c = seed * 0x100000000ULL + (offset + i) * 2ULL;
    float k = k_lo + (k_hi - k_lo) * u01(splitmix64(c));
    float s = u01(splitmix64(c + 1));
    float z = fabsf(1.0f - k) + 2.0f * fminf(k, 1.0f) * s;
    float le, ld, ed;
    pt::ma_terms(k, z, &le, &ld, &ed);
    float ik2 = 1.0f / (k * k);
    if (X) {
        X[2 * i] = (k - norm[0]) / norm[1];
        X[2 * i + 1] = pt::band_coord(s);
    }
    if (T) {
        T[2 * i] = (ld * ik2 - norm[2]) / norm[3];
        T[2 * i + 1] = (ed * ik2 - norm[4]) / norm[5];
    }
    if (kz) {
        kz[2 * i] = k;
        kz[2 * i + 1] = z;
    }
}

// ---------------------------------------------------------------------------
// Tiled FP32 GEMM, C[m][n] = sum_k A(m,k) B(k,n) with strided operands,
// 64 x 64 tile per 256 threads, 4 x 4 per thread, k step 16.
// ---------------------------------------------------------------------------
enum { EPI_PLAIN = 0, EPI_BIAS_SILU = 1, EPI_DSILU = 2 };

struct GemmArgs {
    const float *A;
    long sam, sak;
    const float *B;
    long sbk, sbn;
    int M, N, K;
    int k_chunk;            // split-K: blockIdx.z covers [z*k_chunk, (z+1)*k_chunk)
    float *C;               // [M][N] (+ blockIdx.z * M * N for split-K partials)
    const float *bias;      // EPI_BIAS_SILU
    float *H;               // EPI_BIAS_SILU: silu(C)
    const float *Zaux;      // EPI_DSILU: C = acc * dsilu(Zaux)
    int round_a, round_b;   // round operands to BF16 (quantisation-aware forward)
};

template <int EPI>
__global__ void __launch_bounds__(256) gemm_kernel(GemmArgs g)
{
    __shared__ float As[16][64 + 4];
    __shared__ float Bs[16][64 + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int kb = blockIdx.z * g.k_chunk;
    const int ke = min(g.K, kb + g.k_chunk);
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    for (int k0 = kb; k0 < ke; k0 += 16) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int idx = threadIdx.x + r * 256;        // 0..1023
            int kk = idx & 15, mm = idx >> 4;       // A tile [64][16]
            int gm = m0 + mm, gk = k0 + kk;
            float a = (gm < g.M && gk < ke) ? g.A[gm * g.sam + gk * g.sak] : 0.0f;
            As[kk][mm] = g.round_a ? bf16r(a) : a;
            int nn = idx & 63, kk2 = idx >> 6;      // B tile [16][64]
            int gn = n0 + nn, gk2 = k0 + kk2;
            float b = (gn < g.N && gk2 < ke) ? g.B[gk2 * g.sbk + gn * g.sbn] : 0.0f;
            Bs[kk2][nn] = g.round_b ? bf16r(b) : b;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    float *C = g.C + (size_t)blockIdx.z * g.M * g.N;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int m = m0 + ty * 4 + i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int n = n0 + tx * 4 + j;
            if (n >= g.N) continue;
            float v = acc[i][j];
            if (EPI == EPI_BIAS_SILU) {
                v += g.bias[n];
                g.H[(size_t)m * g.N + n] = silu(v);
            } else if (EPI == EPI_DSILU) {
                v *= dsilu(g.Zaux[(size_t)m * g.N + n]);
            }
            C[(size_t)m * g.N + n] = v;
        }
    }
}

template <int EPI>
int gemm(const GemmArgs &g, int splits, cudaStream_t s)
{
    dim3 grid((g.N + 63) / 64, (g.M + 63) / 64, splits);
    gemm_kernel<EPI><<<grid, 256, 0, s>>>(g);
    return cuda_status("gemm_kernel");
}

// Layer 1 (2 -> 128): Z1 = X W1^T + b1, H1 = silu(Z1).
__global__ void layer1_kernel(const float *p, const float *X, int n, float *Z1, float *H1)
{
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * H) return;
    int i = (int)(idx / H), j = (int)(idx % H);
    float z = fmaf(p[OFF_W1 + 2 * j], X[2 * i], fmaf(p[OFF_W1 + 2 * j + 1], X[2 * i + 1], p[OFF_B1 + j]));
    Z1[idx] = z;
    H1[idx] = silu(z);
}

// Output layer (128 -> 2), loss terms and dZ3 = (dY W4) * silu'(Z3).
// One warp per sample.
__global__ void output_kernel(const float *p, const float *H3, const float *Z3, const float *T, int n, float *Y,
                              float *dY, float *dZ3, float *loss_part)
{
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const float *h = H3 + (size_t)warp * H;
    float a0 = 0.0f, a1 = 0.0f;
    for (int i = lane; i < H; i += 32) {
        a0 = fmaf(p[OFF_W4 + i], h[i], a0);
        a1 = fmaf(p[OFF_W4 + H + i], h[i], a1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    }
    float y0 = a0 + p[OFF_B4], y1 = a1 + p[OFF_B4 + 1];
    float r0 = 0.0f, r1 = 0.0f;
    if (T) {
        r0 = y0 - T[2 * warp];
        r1 = y1 - T[2 * warp + 1];
    }
    float d0 = 2.0f * r0 / (float)n, d1 = 2.0f * r1 / (float)n;
    if (lane == 0) {
        if (Y) {
            Y[2 * warp] = y0;
            Y[2 * warp + 1] = y1;
        }
        if (dY) {
            dY[2 * warp] = d0;
            dY[2 * warp + 1] = d1;
        }
        if (loss_part) loss_part[warp] = r0 * r0 + r1 * r1;
    }
    if (dZ3) {
        for (int i = lane; i < H; i += 32) {
            float dh = p[OFF_W4 + i] * d0 + p[OFF_W4 + H + i] * d1;
            dZ3[(size_t)warp * H + i] = dh * dsilu(Z3[(size_t)warp * H + i]);
        }
    }
}

// Gradient of the output layer and of layer 1, and the bias gradients of
// the hidden layers: deterministic sums over the batch in chunks of SPLIT
// rows.  part layout per chunk: [gW4 (256) | gb4 (2) | gW1 (256) | gb1 (128) |
// gb2 (128) | gb3 (128)] = 898 floats.
constexpr int SMALL = 2 * H + 2 + 2 * H + H + H + H;

__global__ void small_grad_kernel(const float *X, const float *H3, const float *dY, const float *dZ1,
                                  const float *dZ2, const float *dZ3, int n, float *part)
{
    int chunk = blockIdx.x;
    int r0 = chunk * SPLIT, r1 = min(n, r0 + SPLIT);
    float *out = part + (size_t)chunk * SMALL;
    for (int q = threadIdx.x; q < SMALL; q += blockDim.x) {
        float acc = 0.0f;
        if (q < 2 * H) {                          // gW4[o][i]
            int o = q / H, i = q % H;
            for (int r = r0; r < r1; ++r) acc = fmaf(dY[2 * r + o], H3[(size_t)r * H + i], acc);
        } else if (q < 2 * H + 2) {               // gb4
            int o = q - 2 * H;
            for (int r = r0; r < r1; ++r) acc += dY[2 * r + o];
        } else if (q < 4 * H + 2) {               // gW1[j][c]
            int jc = q - (2 * H + 2), j = jc / 2, c = jc % 2;
            for (int r = r0; r < r1; ++r) acc = fmaf(dZ1[(size_t)r * H + j], X[2 * r + c], acc);
        } else {                                  // gb1, gb2, gb3
            int t = q - (4 * H + 2), l = t / H, j = t % H;
            const float *dZ = (l == 0) ? dZ1 : (l == 1) ? dZ2 : dZ3;
            for (int r = r0; r < r1; ++r) acc += dZ[(size_t)r * H + j];
        }
        out[q] = acc;
    }
}

// Sum the split partials in chunk order and scatter into the gradient.
__global__ void reduce_grad_kernel(const float *pw2, const float *pw3, const float *psmall, int nchunk, float *grad)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < H * H) {
        float a = 0.0f, b = 0.0f;
        for (int c = 0; c < nchunk; ++c) {
            a += pw2[(size_t)c * H * H + q];
            b += pw3[(size_t)c * H * H + q];
        }
        grad[OFF_W2 + q] = a;
        grad[OFF_W3 + q] = b;
    }
    if (q < SMALL) {
        float a = 0.0f;
        for (int c = 0; c < nchunk; ++c) a += psmall[(size_t)c * SMALL + q];
        int dst;
        if (q < 2 * H) dst = OFF_W4 + q;
        else if (q < 2 * H + 2) dst = OFF_B4 + (q - 2 * H);
        else if (q < 4 * H + 2) dst = OFF_W1 + (q - (2 * H + 2));
        else {
            int t = q - (4 * H + 2), l = t / H, j = t % H;
            dst = (l == 0 ? OFF_B1 : l == 1 ? OFF_B2 : OFF_B3) + j;
        }
        grad[dst] = a;
    }
}

__global__ void loss_reduce_kernel(const float *part, int n, float *loss)
{
    __shared__ float s[256];
    float a = 0.0f;
    for (int i = threadIdx.x; i < n; i += 256) a += part[i];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = s[0] / (float)n;
}

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

struct Work {
    float *Z1, *H1, *Z2, *H2, *Z3, *H3, *dZ1, *dZ2, *dZ3, *Y, *dY, *lpart, *pw2, *pw3, *psmall;
    size_t bytes;
};

Work carve(void *base, int n)
{
    int nchunk = (n + SPLIT - 1) / SPLIT;
    size_t a = (size_t)n * H;
    Work w;
    char *p = (char *)base;
    size_t off = 0;
    auto take = [&](size_t count) {
        float *r = (float *)(p + off);
        off += ((count * sizeof(float)) + 255) & ~(size_t)255;
        return r;
    };
    w.Z1 = take(a);
    w.H1 = take(a);
    w.Z2 = take(a);
    w.H2 = take(a);
    w.Z3 = take(a);
    w.H3 = take(a);
    w.dZ1 = take(a);
    w.dZ2 = take(a);
    w.dZ3 = take(a);
    w.Y = take((size_t)2 * n);
    w.dY = take((size_t)2 * n);
    w.lpart = take((size_t)n);
    w.pw2 = take((size_t)nchunk * H * H);
    w.pw3 = take((size_t)nchunk * H * H);
    w.psmall = take((size_t)nchunk * SMALL);
    w.bytes = off;
    return w;
}

int forward(const float *p, const float *X, int n, const Work &w, int qat, cudaStream_t s)
{
    layer1_kernel<<<(unsigned)(((size_t)n * H + 255) / 256), 256, 0, s>>>(p, X, n, w.Z1, w.H1);
    int st = cuda_status("layer1_kernel");
    if (st) return st;
    // Z_l = H_{l-1} W_l^T: A(m,k) = H[m*H + k], B(k,n) = W[n*H + k]
    GemmArgs g{};
    g.A = w.H1; g.sam = H; g.sak = 1;
    g.B = p + OFF_W2; g.sbk = 1; g.sbn = H;
    g.M = n; g.N = H; g.K = H; g.k_chunk = H;
    g.C = w.Z2; g.bias = p + OFF_B2; g.H = w.H2;
    g.round_a = qat; g.round_b = qat;
    st = gemm<EPI_BIAS_SILU>(g, 1, s);
    if (st) return st;
    g.A = w.H2; g.B = p + OFF_W3; g.C = w.Z3; g.bias = p + OFF_B3; g.H = w.H3;
    return gemm<EPI_BIAS_SILU>(g, 1, s);
}

}  // namespace

extern "C" {

size_t pt_mlp_work_bytes(int n)
{
    if (n < 1) return 0;
    return carve(nullptr, n).bytes;
}

int pt_mlp_forward(const float *params, const float *X, int n, int qat, float *Y, void *work, size_t work_bytes,
                   pt_stream_t stream)
{
    if (n < 0) return PT_ERR_ARG;
    if (n == 0) return PT_OK;
    if (!params || !X || !Y) return PT_ERR_ARG;
    if (!work || work_bytes < pt_mlp_work_bytes(n)) return PT_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    Work w = carve(work, n);
    int st = forward(params, X, n, w, qat ? 1 : 0, s);
    if (st) return st;
    output_kernel<<<(unsigned)(((size_t)n * 32 + 255) / 256), 256, 0, s>>>(params, w.H3, w.Z3, nullptr, n, Y,
                                                                           nullptr, nullptr, nullptr);
    return cuda_status("output_kernel");
}

int pt_mlp_loss_grad(const float *params, const float *X, const float *T, int n, int qat, float *grad, float *loss,
                     void *work, size_t work_bytes, pt_stream_t stream)
{
    if (n < 1 || !params || !X || !T || !grad || !loss) return PT_ERR_ARG;
    if (!work || work_bytes < pt_mlp_work_bytes(n)) return PT_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    Work w = carve(work, n);
    int st = forward(params, X, n, w, qat ? 1 : 0, s);
    if (st) return st;
    output_kernel<<<(unsigned)(((size_t)n * 32 + 255) / 256), 256, 0, s>>>(params, w.H3, w.Z3, T, n, w.Y, w.dY,
                                                                           w.dZ3, w.lpart);
    st = cuda_status("output_kernel");
    if (st) return st;
    const int nchunk = (n + SPLIT - 1) / SPLIT;
    // dZ2 = (dZ3 W3) * silu'(Z2): A(m,k) = dZ3[m*H + k], B(k,n) = W3[k*H + n]
    GemmArgs g{};
    g.A = w.dZ3; g.sam = H; g.sak = 1;
    g.B = params + OFF_W3; g.sbk = H; g.sbn = 1;
    g.M = n; g.N = H; g.K = H; g.k_chunk = H;
    g.C = w.dZ2; g.Zaux = w.Z2;
    g.round_b = qat ? 1 : 0;
    st = gemm<EPI_DSILU>(g, 1, s);
    if (st) return st;
    g.A = w.dZ2; g.B = params + OFF_W2; g.C = w.dZ1; g.Zaux = w.Z1;
    st = gemm<EPI_DSILU>(g, 1, s);
    if (st) return st;
    // dW_l = dZ_l^T H_{l-1}, split over the batch: A(m,k) = dZ[k*H + m], B(k,n) = Hprev[k*H + n]
    GemmArgs d{};
    d.sam = 1; d.sak = H; d.sbk = H; d.sbn = 1;
    d.M = H; d.N = H; d.K = n; d.k_chunk = SPLIT;
    d.A = w.dZ3; d.B = w.H2; d.C = w.pw3; d.round_b = qat ? 1 : 0;
    st = gemm<EPI_PLAIN>(d, nchunk, s);
    if (st) return st;
    d.A = w.dZ2; d.B = w.H1; d.C = w.pw2;
    st = gemm<EPI_PLAIN>(d, nchunk, s);
    if (st) return st;
    small_grad_kernel<<<nchunk, 256, 0, s>>>(X, w.H3, w.dY, w.dZ1, w.dZ2, w.dZ3, n, w.psmall);
    st = cuda_status("small_grad_kernel");
    if (st) return st;
    reduce_grad_kernel<<<(H * H + 255) / 256, 256, 0, s>>>(w.pw2, w.pw3, w.psmall, nchunk, grad);
    st = cuda_status("reduce_grad_kernel");
    if (st) return st;
    loss_reduce_kernel<<<1, 256, 0, s>>>(w.lpart, n, loss);
    return cuda_status("loss_reduce_kernel");
}

int pt_mlp_adam(float *params, const float *grad, float *m, float *v, int step, float lr, float beta1, float beta2,
                float eps, pt_stream_t stream)
{
    if (!params || !grad || !m || !v || step < 1) return PT_ERR_ARG;
    float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    adam_kernel<<<(NPAR + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, NPAR, lr, beta1, beta2,
                                                                      eps, c1, c2);
    return cuda_status("adam_kernel");
}

int pt_sur_datagen(unsigned long long seed, size_t offset, size_t n, float k_lo, float k_hi, const float *norm,
                   float *X, float *T, float *kz, pt_stream_t stream)
{
    if (n == 0) return PT_OK;
    if (!norm || (!X && !T && !kz) || !(k_lo > 0.0f) || !(k_hi >= k_lo) || k_hi > 1.0f) return PT_ERR_ARG;
    size_t blocks = (n + 255) / 256;
    if (blocks > 0x7fffffffULL) return PT_ERR_ARG;
    datagen_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(seed, offset, n, k_lo, k_hi, norm, X, T, kz);
    return cuda_status("datagen_kernel");
}

}  // extern "C"
