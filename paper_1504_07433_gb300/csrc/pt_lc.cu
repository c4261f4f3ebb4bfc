// pt_lc.cu -- light-curve kernels and their C ABI (include/pt.h).
//
// Kernel structure of the fused light-curve path (Secs. 2.1, 2.2, 3.2, 3.4):
//   setup_kernel   per geometry: FP64 conjunction anchor, double-float t0/P,
//                  a conservative transit window; per time: double-float split.
//   ma_lc_kernel / gim_lc_kernel, one CTA per (256-time tile, VT geometries):
//     A. every (time, geometry) pair: phase reduction + window test; pairs in
//        the window are appended to a shared-memory queue (compaction, so
//        the expensive branches run on full warps);
//     B. queued pairs are expanded to (pair, supersample) units; each unit
//        computes z and the limb-darkening-free terms (lambda_e, lambda_d,
//        eta_d for MA; alpha_0..alpha_N for Gimenez); sums over the
//        supersamples are formed in a fixed order (deterministic);
//     C. every output: the per-passband limb-darkening combination and a
//        coalesced store of the flux cube and/or a deterministic block
//        reduction of the weighted squared residuals.
//   ssr_reduce_kernel: sums the per-tile residual partials in a fixed order.
#include <cuda_runtime.h>

#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/pt.h"
#include "pt_device.cuh"

using pt::GeomRec;

namespace {

constexpr int TT = 256;      // times per CTA (= threads per CTA)
constexpr int VT_MA = 8;     // geometries per CTA, Mandel-Agol
constexpr int VT_G = 2;      // geometries per CTA, Gimenez
constexpr int MAX_SS = 256;  // supersamples per exposure
constexpr int MAX_NEWTON = 64;  // cap on Newton steps
constexpr int G_CHUNK = 64;  // queued pairs per Gimenez evaluation round
constexpr double PI_D = 3.14159265358979323846;

thread_local char g_last_error[512] = "";

int set_cuda_error(cudaError_t e, const char *where)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
    return PT_ERR_CUDA;
}

}  // namespace

// Shared by the other translation units of the library.
namespace pt_internal {
int set_error(int status, const char *where, const char *msg)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, msg);
    return status;
}
}  // namespace pt_internal

namespace {

int check_launch(const char *where)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error(e, where);
    return PT_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// ---------------------------------------------------------------------------
// Set-up kernel
// ---------------------------------------------------------------------------
struct SetupArgs {
    const double *t;
    int n_t;
    float2 *tsplit;
    const double *t0, *P;
    const float *a, *inc, *e, *w, *k;
    int n_v, n_b, k_per_band, n_geom;
    GeomRec *rec;
    float half_exp;
    int n_gblocks;
};

__device__ void make_geom(const SetupArgs &s, int g, GeomRec *out)
{
    int v = s.k_per_band ? g / s.n_b : g;
    pt::make_geom_rec(s.t0[v], s.P[v], s.a[v], s.inc[v], s.e != nullptr, s.e ? s.e[v] : 0.0f,
                      s.w ? s.w[v] : 0.0f, s.k[g], s.half_exp, out);
}

__global__ void setup_kernel(SetupArgs s)
{
    if ((int)blockIdx.x < s.n_gblocks) {
        int g = blockIdx.x * blockDim.x + threadIdx.x;
        if (g < s.n_geom) make_geom(s, g, &s.rec[g]);
    } else {
        int i = (blockIdx.x - s.n_gblocks) * blockDim.x + threadIdx.x;
        if (i < s.n_t) {
            double t = s.t[i];
            float h = (float)t;
            s.tsplit[i] = make_float2(h, (float)(t - (double)h));
        }
    }
}

// ---------------------------------------------------------------------------
// Shared pieces of the light-curve kernels
// ---------------------------------------------------------------------------
struct LcArgs {
    const float2 *tsplit;
    int n_t;
    const GeomRec *rec;
    int n_geom;
    const float *ld;     // [rows][n_ld]
    int n_ld;            // 2 (MA) or N (Gimenez)
    int n_b, k_per_band, n_bpg;
    int n_ss;
    float t_exp;
    int max_iter;
    const float *y, *wt;
    float *flux;
    float *ssr_part;     // [rows][n_tiles]
    int n_tiles;
    int *n_bad;
    // Gimenez
    const float4 *gtab;  // [n_geom][N+1][n_j]: (r1_j, r2_j, r3_{j+1}, T_j)
    int N, n_j;
};

__device__ __forceinline__ float block_sum(float v, float *sred)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sred[warp] = v;
    __syncthreads();
    float tot = 0.0f;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += sred[i];
    }
    return tot;
}

// Phase A, shared by both models: window test + compaction.
template <int VT>
__device__ __forceinline__ void phase_a(const LcArgs &A, GeomRec *srec, float (*sdt)[TT],
                                        unsigned char (*sflag)[TT], unsigned short *squeue, int *sqn)
{
    int tl = threadIdx.x;
    int t = blockIdx.x * TT + tl;
    bool tv = t < A.n_t;
    float2 ts = tv ? A.tsplit[t] : make_float2(0.0f, 0.0f);
    // stage the geometry records (6 float4 each)
    for (int i = tl; i < VT * 6; i += TT) {
        int vl = i / 6, c = i % 6;
        int g = blockIdx.y * VT + vl;
        if (g < A.n_geom)
            reinterpret_cast<float4 *>(&srec[vl])[c] = reinterpret_cast<const float4 *>(&A.rec[g])[c];
    }
    if (tl == 0) *sqn = 0;
    __syncthreads();
#pragma unroll 1
    for (int vl = 0; vl < VT; ++vl) {
        int g = blockIdx.y * VT + vl;
        bool valid = tv && g < A.n_geom;
        float dt = 0.0f;
        bool inw = false;
        if (valid) {
            dt = pt::reduce_time(ts.x, ts.y, srec[vl]);
            inw = (dt >= srec[vl].win_lo) && (dt <= srec[vl].win_hi);
        }
        sdt[vl][tl] = dt;
        sflag[vl][tl] = inw ? 1 : 0;
        int slot = pt::warp_append(sqn, inw);
        if (inw) squeue[slot] = (unsigned short)(vl * TT + tl);
    }
    __syncthreads();
}

__device__ __forceinline__ float ss_offset(float t_exp, int s, int n_ss)
{
    return t_exp * (((float)s + 0.5f) / (float)n_ss - 0.5f);
}

// ---------------------------------------------------------------------------
// Mandel-Agol light curves
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TT) ma_lc_kernel(LcArgs A)
{
    __shared__ GeomRec srec[VT_MA];
    __shared__ float sdt[VT_MA][TT];
    __shared__ unsigned char sflag[VT_MA][TT];
    __shared__ unsigned short squeue[VT_MA * TT];
    __shared__ float sacc[3][VT_MA][TT];
    __shared__ float sub[3][TT];
    __shared__ float sred[TT / 32];
    __shared__ int sqn, sbad;

    if (threadIdx.x == 0) sbad = 0;
    phase_a<VT_MA>(A, srec, sdt, sflag, squeue, &sqn);
    const int tl = threadIdx.x;
    const int qn = sqn;
    const int nss = A.n_ss;
    const int G = TT / nss;
    const int units = G * nss;

    // Phase B: (pair, supersample) units
#pragma unroll 1
    for (int base = 0; base < qn; base += G) {
        int iu = tl / nss;
        int s = tl - iu * nss;
        int item = base + iu;
        float le = 0.0f, ld = 0.0f, ed = 0.0f;
        if (tl < units && item < qn) {
            int code = squeue[item];
            int vl = code / TT, ti = code % TT;
            const GeomRec &r = srec[vl];
            float dts = sdt[vl][ti] + ss_offset(A.t_exp, s, nss);
            bool bad = false;
            float z = pt::orbit_z(r, dts, A.max_iter, &bad);
            if (bad) atomicAdd(&sbad, 1);
            pt::ma_terms(r.k, z, &le, &ld, &ed);
        }
        sub[0][tl] = le;
        sub[1][tl] = ld;
        sub[2][tl] = ed;
        __syncthreads();
        if (tl < G && base + tl < qn) {
            float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
            for (int j = 0; j < nss; ++j) {
                s0 += sub[0][tl * nss + j];
                s1 += sub[1][tl * nss + j];
                s2 += sub[2][tl * nss + j];
            }
            int code = squeue[base + tl];
            int vl = code / TT, ti = code % TT;
            sacc[0][vl][ti] = s0;
            sacc[1][vl][ti] = s1;
            sacc[2][vl][ti] = s2;
        }
        __syncthreads();
    }

    // Phase C: limb darkening per passband, stores and residuals
    const int t = blockIdx.x * TT + tl;
    const bool tv = t < A.n_t;
    const float inv_nss = 1.0f / (float)nss;
#pragma unroll 1
    for (int vl = 0; vl < VT_MA; ++vl) {
        int g = blockIdx.y * VT_MA + vl;
        if (g >= A.n_geom) break;
        bool inw = tv && sflag[vl][tl];
        float l0 = 0.0f, l1 = 0.0f, l2 = 0.0f;
        if (inw) {
            l0 = sacc[0][vl][tl] * inv_nss;
            l1 = sacc[1][vl][tl] * inv_nss;
            l2 = sacc[2][vl][tl] * inv_nss;
        }
#pragma unroll 1
        for (int bb = 0; bb < A.n_bpg; ++bb) {
            int row = g * A.n_bpg + bb;
            float we, wd, wn;
            pt::ma_weights(A.ld[row * 2], A.ld[row * 2 + 1], &we, &wd, &wn);
            float f = inw ? 1.0f - (we * l0 + wd * l1 + wn * l2) : 1.0f;
            if (A.flux && tv) A.flux[(size_t)row * A.n_t + t] = f;
            if (A.ssr_part) {
                int band = A.k_per_band ? (g % A.n_b) : bb;
                float val = 0.0f;
                if (tv) {
                    float r = A.y[(size_t)band * A.n_t + t] - f;
                    val = (A.wt ? A.wt[(size_t)band * A.n_t + t] : 1.0f) * r * r;
                }
                float tot = block_sum(val, sred);
                if (tl == 0) A.ssr_part[(size_t)row * A.n_tiles + blockIdx.x] = tot;
            }
        }
    }
    if (tl == 0 && sbad && A.n_bad) atomicAdd(A.n_bad, sbad);
}

// ---------------------------------------------------------------------------
// Gimenez light curves
//
// Per geometry the set-up pass stores T_{n,j} = A_{n,j} G_j(nu+2, nu+1; 1-b)^2
// (Sec. 2.1.4: the z-independent factors).  Per unit the kernel runs the
// three-term recursion of G_j(nu+2, 1; c^2) and accumulates
//   alpha_n = b^2 (1 - c^2)^{nu+1} sum_j T_{n,j} G_j(nu+2, 1; c^2),
// "only summations and multiplications" (Sec. 2.1.4).  Units are
// (pair, n) so that a warp shares n (broadcast coefficient loads); each unit
// carries all supersamples of its pair in registers, SB at a time.
// ---------------------------------------------------------------------------
template <int SB>
__device__ __forceinline__ void gim_unit(const float4 *tab, int n_j, int n, float b2, const float *sx,
                                         const float *sq, int nss, float *acc_out)
{
    // Clenshaw's backward summation of S = sum_j T_j G_j with
    // G_{j+1} = (r1_j + r2_j x) G_j + r3_j G_{j-1}, G_0 = 1, G_{-1} = 0:
    //   b_j = T_j + (r1_j + r2_j x) b_{j+1} + r3_{j+1} b_{j+2},  S = b_0,
    // three FMAs per term; tab[j] = (r1_j, r2_j, r3_{j+1}, T_j).
    float acc = 0.0f;
#pragma unroll 1
    for (int s0 = 0; s0 < nss; s0 += SB) {
        float x[SB], b1[SB], b2v[SB];
        bool any = false;
#pragma unroll
        for (int u = 0; u < SB; ++u) {
            int s = s0 + u;
            x[u] = (s < nss) ? sx[s] : 0.0f;
            any |= (s < nss) && (sq[s] > 0.0f);
            b1[u] = 0.0f;
            b2v[u] = 0.0f;
        }
        if (!any) continue;   // every supersample of this block is out of transit
#pragma unroll 2
        for (int j = n_j - 1; j >= 0; --j) {
            float4 c = tab[j];
#pragma unroll
            for (int u = 0; u < SB; ++u) {
                float al = fmaf(c.y, x[u], c.x);
                float t = fmaf(c.z, b2v[u], c.w);
                float bj = fmaf(al, b1[u], t);
                b2v[u] = b1[u];
                b1[u] = bj;
            }
        }
#pragma unroll
        for (int u = 0; u < SB; ++u) {
            int s = s0 + u;
            if (s < nss) {
                // (1 - c^2)^{nu+1} = (1 - c^2)^2 sqrt(1 - c^2)^n, nu = (n+2)/2
                float q = sq[s];
                float q2 = q * q;
                float pw = q2 * q2;
                for (int i = 0; i < n; ++i) pw *= q;
                acc = fmaf(b2 * pw, b1[u], acc);
            }
        }
    }
    *acc_out = acc;
}

template <int SB>
__global__ void __launch_bounds__(TT) gim_lc_kernel(LcArgs A)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ GeomRec srec[VT_G];
    __shared__ float sdt[VT_G][TT];
    __shared__ unsigned char sflag[VT_G][TT];
    __shared__ unsigned short squeue[VT_G * TT];
    __shared__ float sred[TT / 32];
    __shared__ int sqn, sbad;

    const int NP1 = A.N + 1;
    const int nj = A.n_j;
    float4 *stab = reinterpret_cast<float4 *>(dsm);                    // [VT_G][NP1][nj]
    float *sacc = reinterpret_cast<float *>(stab + VT_G * NP1 * nj);   // [VT_G][NP1][TT]
    float *sx = sacc + VT_G * NP1 * TT;                                 // [G_CHUNK][n_ss]
    float *sq = sx + G_CHUNK * A.n_ss;                                  // [G_CHUNK][n_ss]

    if (threadIdx.x == 0) sbad = 0;
    phase_a<VT_G>(A, srec, sdt, sflag, squeue, &sqn);
    const int tl = threadIdx.x;
    const int qn = sqn;
    const int nss = A.n_ss;

    if (qn > 0) {
        for (int vl = 0; vl < VT_G; ++vl) {
            int g = blockIdx.y * VT_G + vl;
            if (g >= A.n_geom) break;
            const float4 *src = A.gtab + (size_t)g * NP1 * nj;
            for (int i = tl; i < NP1 * nj; i += TT) stab[vl * NP1 * nj + i] = src[i];
        }
    }
    __syncthreads();

#pragma unroll 1
    for (int base = 0; base < qn; base += G_CHUNK) {
        int nit = min(G_CHUNK, qn - base);
        // B1: z of every (pair, supersample) of the chunk
        for (int u = tl; u < nit * nss; u += TT) {
            int il = u / nss, s = u - il * nss;
            int code = squeue[base + il];
            int vl = code / TT, ti = code % TT;
            const GeomRec &r = srec[vl];
            float dts = sdt[vl][ti] + ss_offset(A.t_exp, s, nss);
            bool bad = false;
            float z = pt::orbit_z(r, dts, A.max_iter, &bad);
            if (bad) atomicAdd(&sbad, 1);
            float xv = 0.0f, qv = 0.0f;
            if (z < 1.0f + r.k) {
                float c = z / (1.0f + r.k);
                xv = c * c;
                qv = sqrtf((1.0f - c) * (1.0f + c));
            }
            sx[u] = xv;
            sq[u] = qv;
        }
        __syncthreads();
        // B2: (pair, n) units
        for (int u = tl; u < nit * NP1; u += TT) {
            int n = u / nit, il = u - n * nit;
            int code = squeue[base + il];
            int vl = code / TT, ti = code % TT;
            float kk = srec[vl].k;
            float bb = kk / (1.0f + kk);
            float acc;
            gim_unit<SB>(stab + (vl * NP1 + n) * nj, nj, n, bb * bb, sx + il * nss, sq + il * nss, nss, &acc);
            sacc[(vl * NP1 + n) * TT + ti] = acc;
        }
        __syncthreads();
    }

    // Phase C
    const int t = blockIdx.x * TT + tl;
    const bool tv = t < A.n_t;
    const float inv_nss = 1.0f / (float)nss;
#pragma unroll 1
    for (int vl = 0; vl < VT_G; ++vl) {
        int g = blockIdx.y * VT_G + vl;
        if (g >= A.n_geom) break;
        bool inw = tv && sflag[vl][tl];
#pragma unroll 1
        for (int bb = 0; bb < A.n_bpg; ++bb) {
            int row = g * A.n_bpg + bb;
            const float *u = A.ld + (size_t)row * A.N;
            float f = 1.0f;
            if (inw) {
                // C_0 = (1 - sum u)/D, C_n = u_n/D, D = 1 - sum n u_n/(n+2)   (Sec. 2.1.3)
                float su = 0.0f, sd = 0.0f;
                for (int n = 1; n <= A.N; ++n) {
                    float un = u[n - 1];
                    su += un;
                    sd += (float)n * un / (float)(n + 2);
                }
                float invD = 1.0f / (1.0f - sd);
                float al = (1.0f - su) * sacc[(vl * NP1 + 0) * TT + tl];
                for (int n = 1; n <= A.N; ++n) al = fmaf(u[n - 1], sacc[(vl * NP1 + n) * TT + tl], al);
                f = 1.0f - al * invD * inv_nss;
            }
            if (A.flux && tv) A.flux[(size_t)row * A.n_t + t] = f;
            if (A.ssr_part) {
                int band = A.k_per_band ? (g % A.n_b) : bb;
                float val = 0.0f;
                if (tv) {
                    float r = A.y[(size_t)band * A.n_t + t] - f;
                    val = (A.wt ? A.wt[(size_t)band * A.n_t + t] : 1.0f) * r * r;
                }
                float tot = block_sum(val, sred);
                if (tl == 0) A.ssr_part[(size_t)row * A.n_tiles + blockIdx.x] = tot;
            }
        }
    }
    if (tl == 0 && sbad && A.n_bad) atomicAdd(A.n_bad, sbad);
}

size_t gim_dyn_smem(int N, int n_j, int n_ss)
{
    int NP1 = N + 1;
    size_t b = (size_t)VT_G * NP1 * n_j * sizeof(float4);
    b += (size_t)VT_G * NP1 * TT * sizeof(float);
    b += (size_t)2 * G_CHUNK * n_ss * sizeof(float);
    return b;
}

// Gimenez per-geometry table for Clenshaw's summation: entry (n, j) packs the
// z-recursion coefficients r1_j, r2_j, r3_{j+1} of G_j(nu+2, 1; x) with
// T_{n,j} = A_{n,j} G_j(nu+2, nu+1; 1-b)^2, the z-independent factor of
// Sec. 2.1.4 (FP64 recursion, stored FP32).
__global__ void gim_table_kernel(const GeomRec *rec, int n_geom, int NP1, int n_j, const double *A,
                                 const double *recb, const float4 *coef, float4 *tab)
{
    int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n_geom * NP1) return;
    int g = id / NP1, n = id % NP1;
    double k = rec[g].k;
    double x = 1.0 - k / (1.0 + k);
    const double *An = A + (size_t)n * n_j;
    const double *rb = recb + (size_t)n * n_j * 3;
    const float4 *cf = coef + (size_t)n * n_j;
    float4 *out = tab + ((size_t)g * NP1 + n) * n_j;
    double gp = 0.0, gc = 1.0;
    for (int j = 0; j < n_j; ++j) {
        float4 c = cf[j];
        float r3n = (j + 1 < n_j) ? cf[j + 1].z : 0.0f;
        out[j] = make_float4(c.x, c.y, r3n, (float)(An[j] * gc * gc));
        double gn = (rb[3 * j] + rb[3 * j + 1] * x) * gc + rb[3 * j + 2] * gp;
        gp = gc;
        gc = gn;
    }
}

__global__ void ssr_reduce_kernel(const float *part, int rows, int n_tiles, float *ssr)
{
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= rows) return;
    float s = 0.0f;
    for (int i = lane; i < n_tiles; i += 32) s += part[(size_t)warp * n_tiles + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) ssr[warp] = s;
}

// ---------------------------------------------------------------------------
// Pointwise kernels
// ---------------------------------------------------------------------------
__global__ void ma_terms_kernel(const float *k, const float *z, size_t n, float *le, float *ld, float *ed)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float a, b, c;
    pt::ma_terms(k[i], fabsf(z[i]), &a, &b, &c);
    if (le) le[i] = a;
    if (ld) ld[i] = b;
    if (ed) ed[i] = c;
}

__global__ void gim_alpha_kernel(const float *kk, const float *zz, size_t n, int NP1, int n_j,
                                 const float4 *coef, const double *A, const double *recb, float *alpha)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float k = kk[i], z = fabsf(zz[i]);
    float *out = alpha + i * NP1;
    if (!(z < 1.0f + k) || !(k > 0.0f)) {
        for (int m = 0; m < NP1; ++m) out[m] = 0.0f;
        return;
    }
    float c = z / (1.0f + k);
    float x = c * c;
    float q = sqrtf((1.0f - c) * (1.0f + c));
    float bb = k / (1.0f + k);
    double xb = 1.0 - (double)k / (1.0 + (double)k);
    for (int n = 0; n < NP1; ++n) {
        const double *An = A + (size_t)n * n_j;
        const double *rb = recb + (size_t)n * n_j * 3;
        const float4 *cf = coef + (size_t)n * n_j;
        double hp = 0.0, hc = 1.0;
        float g = 1.0f, gp = 0.0f;
        float sum = (float)An[0];
        for (int j = 0; j + 1 < n_j; ++j) {
            double hn = (rb[3 * j] + rb[3 * j + 1] * xb) * hc + rb[3 * j + 2] * hp;
            hp = hc;
            hc = hn;
            float tj = (float)(An[j + 1] * hc * hc);
            float4 cc = cf[j];
            float gn = fmaf(fmaf(cc.y, x, cc.x), g, cc.z * gp);
            gp = g;
            g = gn;
            sum = fmaf(tj, gn, sum);
        }
        float q2 = q * q, pw = q2 * q2;
        for (int m = 0; m < n; ++m) pw *= q;
        out[n] = bb * bb * pw * sum;
    }
}

// ---------------------------------------------------------------------------
// z kernels (standalone)
// ---------------------------------------------------------------------------
__global__ void z_circ_kernel(const double *t, int n_t, const double *t0, const double *P, const float *a,
                              const float *inc, int n_ss, double t_exp, float *z)
{
    int v = blockIdx.y;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_t * n_ss) return;
    int i = idx / n_ss, s = idx - i * n_ss;
    double tt = t[i] + t_exp * ((s + 0.5) / n_ss - 0.5);
    double x = (tt - t0[v]) * (1.0 / P[v]);
    x -= rint(x);
    float ph = (float)(2.0 * PI_D * x);
    float sp, cp;
    sincosf(ph, &sp, &cp);
    float out = PT_ZBEHIND;
    if (cp > 0.0f) {
        float ci = (float)cos((double)inc[v]) * cp;
        out = a[v] * sqrtf(fmaf(sp, sp, ci * ci));
    }
    z[(size_t)v * n_t * n_ss + idx] = out;
}

__global__ void z_ecc_kernel(const double *t, int n_t, const double *t0, const double *P, const float *a,
                             const float *inc, const float *e, const float *w, int n_ss, double t_exp,
                             int max_iter, double tol, float *z, int *n_bad)
{
    __shared__ double sMtr;
    int v = blockIdx.y;
    double ev = e[v], wv = w[v];
    if (threadIdx.x == 0) {
        double ftr = 0.5 * PI_D - wv;
        double Etr = 2.0 * atan2(sqrt(1.0 - ev) * sin(0.5 * ftr), sqrt(1.0 + ev) * cos(0.5 * ftr));
        sMtr = Etr - ev * sin(Etr);
    }
    __syncthreads();
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_t * n_ss) return;
    int i = idx / n_ss, s = idx - i * n_ss;
    double tt = t[i] + t_exp * ((s + 0.5) / n_ss - 0.5);
    double x = (tt - t0[v]) / P[v];
    x -= floor(x);
    double M = sMtr + 2.0 * PI_D * x;
    M -= 2.0 * PI_D * floor(M / (2.0 * PI_D));
    // FP64 Newton iteration on E - e sin E = M, start E = M (e < 0.8) or pi
    double E = (ev < 0.8) ? M : PI_D;
    bool conv = false;
    for (int it = 0; it < max_iter; ++it) {
        double sE, cE;
        sincos(E, &sE, &cE);
        double d = (E - ev * sE - M) / (1.0 - ev * cE);
        E -= d;
        if (fabs(d) < tol) {
            conv = true;
            break;
        }
    }
    if (!conv && n_bad) atomicAdd(n_bad, 1);
    double f = 2.0 * atan2(sqrt(1.0 + ev) * sin(0.5 * E), sqrt(1.0 - ev) * cos(0.5 * E));
    double r = a[v] * (1.0 - ev * cos(E));
    double sw, cw;
    sincos(wv + f, &sw, &cw);
    float out = PT_ZBEHIND;
    if (sw > 0.0) {
        double ci = cos((double)inc[v]);
        out = (float)(r * sqrt(cw * cw + sw * sw * ci * ci));
    }
    z[(size_t)v * n_t * n_ss + idx] = out;
}

int check_orbit(const pt_orbit *orb, bool need_ecc)
{
    if (!orb || orb->n_v < 0) return PT_ERR_ARG;
    if (orb->n_v == 0) return PT_OK;
    if (!orb->t0 || !orb->P || !orb->a || !orb->inc) return PT_ERR_ARG;
    if ((orb->e == nullptr) != (orb->w == nullptr)) return PT_ERR_ARG;
    if (need_ecc && !orb->e) return PT_ERR_ARG;
    return PT_OK;
}

struct WorkLayout {
    size_t rec, tsplit, T, part, total;
};

WorkLayout work_layout(int n_t, int n_v, int n_b, int k_per_band, int NP1, int n_j)
{
    int n_geom = k_per_band ? n_v * n_b : n_v;
    int n_tiles = (n_t + TT - 1) / TT;
    WorkLayout L;
    size_t off = 0;
    L.rec = off;
    off += align256((size_t)n_geom * sizeof(GeomRec));
    L.tsplit = off;
    off += align256((size_t)n_t * sizeof(float2));
    L.T = off;
    off += align256((size_t)n_geom * NP1 * n_j * sizeof(float4));
    L.part = off;
    off += align256((size_t)n_v * n_b * n_tiles * sizeof(float));
    L.total = off;
    return L;
}

}  // namespace

struct pt_gim_plan_s {
    int N, n_j;
    float4 *d_coef;   // [N+1][n_j]: recursion of G_j(nu+2, 1; x), FP32
    double *d_A;      // [N+1][n_j]: A_{n,j}, FP64
    double *d_recb;   // [N+1][n_j][3]: recursion of G_j(nu+2, nu+1; x), FP64
};

namespace {

// Three-term recursion of G_j(p,q;x) = 2F1(-j, p+j; q; x) in the form of
// Sec. 2.1.4, G_{j+1} = ((j1 + j2 x) G_j + j3 G_{j-1}) / j4, written as
// G_{j+1} = (r1 + r2 x) G_j + r3 G_{j-1}.  Entry 0 produces
// G_1 = 1 - (p+1) x / q from G_0 = 1.  For j >= 1, with s = 2j + p (from the
// standard recurrence of the Jacobi polynomial P_j^{(q-1, p-q)}(1 - 2x),
// rescaled by j!/(q)_j):
//   j1 = s [(s+1)(s-1) + (q-1)^2 - (p-q)^2],  j2 = -2 s (s+1)(s-1),
//   j3 = -2 j (j+p-q)(s+1),                    j4 = 2 (j+p)(s-1)(q+j).
void jacobi_rec(double p, double q, int j, double *r)
{
    if (j == 0) {
        r[0] = 1.0;
        r[1] = -(p + 1.0) / q;
        r[2] = 0.0;
        return;
    }
    double s = 2.0 * j + p;
    double j1 = s * ((s + 1.0) * (s - 1.0) + (q - 1.0) * (q - 1.0) - (p - q) * (p - q));
    double j2 = -2.0 * s * (s + 1.0) * (s - 1.0);
    double j3 = -2.0 * j * (j + p - q) * (s + 1.0);
    double j4 = 2.0 * (j + p) * (s - 1.0) * (q + j);
    r[0] = j1 / j4;
    r[1] = j2 / j4;
    r[2] = j3 / j4;
}

}  // namespace

namespace {
template <int SB>
int launch_gim(const LcArgs &A, dim3 grid, size_t smem, cudaStream_t s)
{
    static thread_local size_t configured = 0;
    if (smem > 48 * 1024 && smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(gim_lc_kernel<SB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return set_cuda_error(e, "gim_lc_kernel smem attribute");
        configured = smem;
    }
    gim_lc_kernel<SB><<<grid, TT, smem, s>>>(A);
    return check_launch("gim_lc_kernel");
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int pt_version(void) { return 100; }

const char *pt_status_string(int s)
{
    switch (s) {
    case PT_OK: return "ok";
    case PT_ERR_ARG: return "invalid argument";
    case PT_ERR_DOMAIN: return "parameter outside the supported domain";
    case PT_ERR_NOT_CONVERGED: return "iteration did not converge";
    case PT_ERR_CUDA: return "CUDA error";
    case PT_ERR_WORKSPACE: return "work buffer missing or too small";
    default: return "unknown status";
    }
}

const char *pt_last_error_string(void) { return g_last_error; }

int pt_z_circ(const double *t, int n_t, const pt_orbit *orb, int n_ss, double t_exp, float *z,
              pt_stream_t stream)
{
    int st = check_orbit(orb, false);
    if (st) return st;
    if (n_t < 0 || n_ss < 1 || (n_t > 0 && (!t || !z))) return PT_ERR_ARG;
    if (n_t == 0 || orb->n_v == 0) return PT_OK;
    if ((long long)n_t * n_ss > 0x7fffffffLL || orb->n_v > 65535) return PT_ERR_ARG;
    dim3 grid((n_t * n_ss + 255) / 256, orb->n_v);
    z_circ_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(t, n_t, orb->t0, orb->P, orb->a, orb->inc, n_ss,
                                                           t_exp, z);
    return check_launch("pt_z_circ");
}

int pt_z_ecc(const double *t, int n_t, const pt_orbit *orb, int n_ss, double t_exp, int max_iter, double tol,
             float *z, int *n_bad, pt_stream_t stream)
{
    int st = check_orbit(orb, true);
    if (st) return st;
    if (n_t < 0 || n_ss < 1 || max_iter < 1 || max_iter > 1000 || !(tol > 0.0) || (n_t > 0 && (!t || !z)))
        return PT_ERR_ARG;
    if (n_t == 0 || orb->n_v == 0) return PT_OK;
    if ((long long)n_t * n_ss > 0x7fffffffLL || orb->n_v > 65535) return PT_ERR_ARG;
    dim3 grid((n_t * n_ss + 255) / 256, orb->n_v);
    z_ecc_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(t, n_t, orb->t0, orb->P, orb->a, orb->inc, orb->e,
                                                          orb->w, n_ss, t_exp, max_iter, tol, z, n_bad);
    return check_launch("pt_z_ecc");
}

int pt_ma_terms(const float *k, const float *z, size_t n, float *le, float *ld, float *ed, pt_stream_t stream)
{
    if (n == 0) return PT_OK;
    if (!k || !z) return PT_ERR_ARG;
    size_t blocks = (n + 255) / 256;
    if (blocks > 0x7fffffffULL) return PT_ERR_ARG;
    ma_terms_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(k, z, n, le, ld, ed);
    return check_launch("pt_ma_terms");
}

static int lc_common_check(const double *t, int n_t, const pt_orbit *orb, const float *k, int k_per_band,
                           const float *ld, int n_b, int n_ss, int max_iter, const float *y, float *flux,
                           float *ssr, void *work)
{
    int st = check_orbit(orb, false);
    if (st) return st;
    if (n_t < 0 || n_b < 1 || n_ss < 1 || n_ss > MAX_SS || max_iter < 1 || max_iter > MAX_NEWTON)
        return PT_ERR_ARG;
    if (k_per_band != 0 && k_per_band != 1) return PT_ERR_ARG;
    if (n_t == 0 || orb->n_v == 0) return PT_OK;   // nothing to evaluate
    if (!flux && !ssr) return PT_ERR_ARG;
    if (!t || !k || !ld) return PT_ERR_ARG;
    if (ssr && !y) return PT_ERR_ARG;
    if (!work) return PT_ERR_WORKSPACE;
    return PT_OK;
}

size_t pt_ma_quad_work_bytes(int n_t, int n_v, int n_b, int k_per_band)
{
    if (n_t < 0 || n_v < 0 || n_b < 1) return 0;
    return work_layout(n_t, n_v, n_b, k_per_band, 0, 0).total;
}

static int launch_setup(const double *t, int n_t, const pt_orbit *orb, const float *k, int k_per_band, int n_b,
                        double t_exp, GeomRec *rec, float2 *tsplit, cudaStream_t s)
{
    SetupArgs sa;
    sa.t = t;
    sa.n_t = n_t;
    sa.tsplit = tsplit;
    sa.t0 = orb->t0;
    sa.P = orb->P;
    sa.a = orb->a;
    sa.inc = orb->inc;
    sa.e = orb->e;
    sa.w = orb->w;
    sa.k = k;
    sa.n_v = orb->n_v;
    sa.n_b = n_b;
    sa.k_per_band = k_per_band;
    sa.n_geom = k_per_band ? orb->n_v * n_b : orb->n_v;
    sa.rec = rec;
    sa.half_exp = (float)(0.5 * t_exp);
    const int bs = 64;
    sa.n_gblocks = (sa.n_geom + bs - 1) / bs;
    int n_tblocks = (n_t + bs - 1) / bs;
    setup_kernel<<<sa.n_gblocks + n_tblocks, bs, 0, s>>>(sa);
    return check_launch("setup_kernel");
}

int pt_ma_quad(const double *t, int n_t, const pt_orbit *orb, const float *k, int k_per_band, const float *ld,
               int n_b, int n_ss, double t_exp, int max_iter, const float *y, const float *wt, float *flux,
               float *ssr, void *work, size_t work_bytes, int *n_bad, pt_stream_t stream)
{
    int st = lc_common_check(t, n_t, orb, k, k_per_band, ld, n_b, n_ss, max_iter, y, flux, ssr, work);
    if (st) return st;
    if (n_t == 0 || orb->n_v == 0) return PT_OK;
    WorkLayout L = work_layout(n_t, orb->n_v, n_b, k_per_band, 0, 0);
    if (work_bytes < L.total) return PT_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    char *wb = (char *)work;
    GeomRec *rec = (GeomRec *)(wb + L.rec);
    float2 *tsplit = (float2 *)(wb + L.tsplit);
    float *part = (float *)(wb + L.part);
    st = launch_setup(t, n_t, orb, k, k_per_band, n_b, t_exp, rec, tsplit, s);
    if (st) return st;
    LcArgs A;
    memset(&A, 0, sizeof(A));
    A.tsplit = tsplit;
    A.n_t = n_t;
    A.rec = rec;
    A.n_geom = k_per_band ? orb->n_v * n_b : orb->n_v;
    A.ld = ld;
    A.n_ld = 2;
    A.n_b = n_b;
    A.k_per_band = k_per_band;
    A.n_bpg = k_per_band ? 1 : n_b;
    A.n_ss = n_ss;
    A.t_exp = (float)t_exp;
    A.max_iter = max_iter;
    A.y = y;
    A.wt = wt;
    A.flux = flux;
    A.ssr_part = ssr ? part : nullptr;
    A.n_tiles = (n_t + TT - 1) / TT;
    A.n_bad = n_bad;
    int gy = (A.n_geom + VT_MA - 1) / VT_MA;
    if (gy > 65535) return PT_ERR_ARG;
    dim3 grid(A.n_tiles, gy);
    ma_lc_kernel<<<grid, TT, 0, s>>>(A);
    st = check_launch("ma_lc_kernel");
    if (st) return st;
    if (ssr) {
        int rows = orb->n_v * n_b;
        ssr_reduce_kernel<<<(rows * 32 + 255) / 256, 256, 0, s>>>(part, rows, A.n_tiles, ssr);
        st = check_launch("ssr_reduce_kernel");
    }
    return st;
}

int pt_gim_plan_create(int N, int n_j, pt_gim_plan *out)
{
    if (!out || N < 1 || N > 16 || n_j < 2 || n_j > 512) return PT_ERR_ARG;
    *out = nullptr;
    int NP1 = N + 1;
    size_t cnt = (size_t)NP1 * n_j;
    float4 *hcoef = new float4[cnt];
    double *hA = new double[cnt];
    double *hrb = new double[cnt * 3];
    for (int n = 0; n < NP1; ++n) {
        double nu = 0.5 * (n + 2);
        // A_{n,j} = (-1)^j (2j+nu+2)/nu * prod_{i=1..j} (nu+i)/(i+1)   (Eq. gimemez_a)
        double prod = 1.0;
        for (int j = 0; j < n_j; ++j) {
            if (j > 0) prod *= (nu + j) / (j + 1.0);
            hA[(size_t)n * n_j + j] = ((j & 1) ? -1.0 : 1.0) * (2.0 * j + nu + 2.0) / nu * prod;
            double r[3];
            jacobi_rec(nu + 2.0, 1.0, j, r);
            hcoef[(size_t)n * n_j + j] = make_float4((float)r[0], (float)r[1], (float)r[2], 0.0f);
            jacobi_rec(nu + 2.0, nu + 1.0, j, r);
            for (int c = 0; c < 3; ++c) hrb[((size_t)n * n_j + j) * 3 + c] = r[c];
        }
    }
    pt_gim_plan p = new pt_gim_plan_s;
    p->N = N;
    p->n_j = n_j;
    p->d_coef = nullptr;
    p->d_A = nullptr;
    p->d_recb = nullptr;
    cudaError_t e = cudaMalloc(&p->d_coef, cnt * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_A, cnt * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_recb, cnt * 3 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(p->d_coef, hcoef, cnt * sizeof(float4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_A, hA, cnt * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_recb, hrb, cnt * 3 * sizeof(double), cudaMemcpyHostToDevice);
    delete[] hcoef;
    delete[] hA;
    delete[] hrb;
    if (e != cudaSuccess) {
        cudaFree(p->d_coef);
        cudaFree(p->d_A);
        cudaFree(p->d_recb);
        delete p;
        return set_cuda_error(e, "pt_gim_plan_create");
    }
    *out = p;
    return PT_OK;
}

int pt_gim_plan_destroy(pt_gim_plan p)
{
    if (!p) return PT_OK;
    cudaFree(p->d_coef);
    cudaFree(p->d_A);
    cudaFree(p->d_recb);
    delete p;
    return PT_OK;
}

int pt_gimenez_alpha(pt_gim_plan plan, const float *k, const float *z, size_t n, float *alpha,
                     pt_stream_t stream)
{
    if (!plan) return PT_ERR_ARG;
    if (n == 0) return PT_OK;
    if (!k || !z || !alpha) return PT_ERR_ARG;
    size_t blocks = (n + 127) / 128;
    if (blocks > 0x7fffffffULL) return PT_ERR_ARG;
    gim_alpha_kernel<<<(unsigned)blocks, 128, 0, (cudaStream_t)stream>>>(k, z, n, plan->N + 1, plan->n_j,
                                                                         plan->d_coef, plan->d_A,
                                                                         plan->d_recb, alpha);
    return check_launch("pt_gimenez_alpha");
}

size_t pt_gimenez_work_bytes(pt_gim_plan plan, int n_t, int n_v, int n_b, int k_per_band)
{
    if (!plan || n_t < 0 || n_v < 0 || n_b < 1) return 0;
    return work_layout(n_t, n_v, n_b, k_per_band, plan->N + 1, plan->n_j).total;
}

int pt_gimenez(pt_gim_plan plan, const double *t, int n_t, const pt_orbit *orb, const float *k, int k_per_band,
               const float *ld, int n_b, int n_ss, double t_exp, int max_iter, const float *y, const float *wt,
               float *flux, float *ssr, void *work, size_t work_bytes, int *n_bad, pt_stream_t stream)
{
    if (!plan) return PT_ERR_ARG;
    int st = lc_common_check(t, n_t, orb, k, k_per_band, ld, n_b, n_ss, max_iter, y, flux, ssr, work);
    if (st) return st;
    if (n_t == 0 || orb->n_v == 0) return PT_OK;
    int NP1 = plan->N + 1;
    WorkLayout L = work_layout(n_t, orb->n_v, n_b, k_per_band, NP1, plan->n_j);
    if (work_bytes < L.total) return PT_ERR_WORKSPACE;
    size_t smem = gim_dyn_smem(plan->N, plan->n_j, n_ss);
    if (smem > 200 * 1024) return PT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    char *wb = (char *)work;
    GeomRec *rec = (GeomRec *)(wb + L.rec);
    float2 *tsplit = (float2 *)(wb + L.tsplit);
    float4 *T = (float4 *)(wb + L.T);
    float *part = (float *)(wb + L.part);
    st = launch_setup(t, n_t, orb, k, k_per_band, n_b, t_exp, rec, tsplit, s);
    if (st) return st;
    int n_geom = k_per_band ? orb->n_v * n_b : orb->n_v;
    int tot = n_geom * NP1;
    // FP64 recursion chains: small blocks spread them over many SMs
    gim_table_kernel<<<(tot + 15) / 16, 16, 0, s>>>(rec, n_geom, NP1, plan->n_j, plan->d_A, plan->d_recb,
                                                   plan->d_coef, T);
    st = check_launch("gim_table_kernel");
    if (st) return st;
    LcArgs A;
    memset(&A, 0, sizeof(A));
    A.tsplit = tsplit;
    A.n_t = n_t;
    A.rec = rec;
    A.n_geom = n_geom;
    A.ld = ld;
    A.n_ld = plan->N;
    A.n_b = n_b;
    A.k_per_band = k_per_band;
    A.n_bpg = k_per_band ? 1 : n_b;
    A.n_ss = n_ss;
    A.t_exp = (float)t_exp;
    A.max_iter = max_iter;
    A.y = y;
    A.wt = wt;
    A.flux = flux;
    A.ssr_part = ssr ? part : nullptr;
    A.n_tiles = (n_t + TT - 1) / TT;
    A.n_bad = n_bad;
    A.gtab = T;
    A.N = plan->N;
    A.n_j = plan->n_j;
    int gy = (n_geom + VT_G - 1) / VT_G;
    if (gy > 65535) return PT_ERR_ARG;
    dim3 grid(A.n_tiles, gy);
    if (n_ss % 5 == 0)
        st = launch_gim<5>(A, grid, smem, s);
    else if (n_ss % 4 == 0)
        st = launch_gim<4>(A, grid, smem, s);
    else if (n_ss % 2 == 0)
        st = launch_gim<2>(A, grid, smem, s);
    else if (n_ss == 1)
        st = launch_gim<1>(A, grid, smem, s);
    else
        st = launch_gim<4>(A, grid, smem, s);
    if (st) return st;
    if (ssr) {
        int rows = orb->n_v * n_b;
        ssr_reduce_kernel<<<(rows * 32 + 255) / 256, 256, 0, s>>>(part, rows, A.n_tiles, ssr);
        st = check_launch("ssr_reduce_kernel");
    }
    return st;
}

}  // extern "C"

// ===========================================================================
// Allocation-free variant of pt_ma_quad.
//
// Some callers cannot call cudaMalloc: a host program that hands all device
// memory to its own fixed pool and forbids outside allocations, or a tight
// sampling loop where an allocation (and the stall it can cause) is not
// acceptable.  For them pt_ma_quad_noalloc takes its scratch from a
// statically sized __device__ array instead of a caller-provided work
// buffer.  The array is part of the module image: every GPU that loads the
// library holds PT_MA_NOALLOC_SCRATCH_BYTES of it until the process exits.
// ===========================================================================
namespace {

static __device__ __align__(256) unsigned char g_ma_noalloc_scratch[PT_MA_NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
void *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};
std::mutex g_noalloc_mutex;

// Device address of the scratch array for the current device.  In host code
// the symbol name is only a host-side stand-in, so the address is fetched
// with cudaGetSymbolAddress once per device (with that device current) and
// cached.
int noalloc_scratch(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_cuda_error(e, "pt_ma_quad_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        snprintf(g_last_error, sizeof(g_last_error), "pt_ma_quad_noalloc: device %d beyond the %d supported", dev,
                 NOALLOC_MAX_DEVICES);
        return PT_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_ma_noalloc_scratch);
        if (e != cudaSuccess) return set_cuda_error(e, "pt_ma_quad_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return PT_OK;
}

}  // namespace

extern "C" int pt_ma_quad_noalloc(const double *t, int n_t, const pt_orbit *orb, const float *k, int k_per_band,
                                  const float *ld, int n_b, int n_ss, double t_exp, int max_iter,
                                  const float *y, const float *wt, float *flux, float *ssr, int *n_bad,
                                  pt_stream_t stream)
{
    if (!orb || n_t < 0 || orb->n_v < 0 || n_b < 1) return PT_ERR_ARG;
    size_t need = pt_ma_quad_work_bytes(n_t, orb->n_v, n_b, k_per_band);
    if (need > (size_t)PT_MA_NOALLOC_SCRATCH_BYTES) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "pt_ma_quad_noalloc: this problem needs %zu bytes of scratch, the static scratch holds %zu; "
                 "use pt_ma_quad with a work buffer", need, (size_t)PT_MA_NOALLOC_SCRATCH_BYTES);
        return PT_ERR_WORKSPACE;
    }
    void *scratch = nullptr;
    int st = noalloc_scratch(&scratch);
    if (st) return st;
    // Every scratch byte the kernels read is written earlier in the same call
    // (geometry records, time split, residual partials), so nothing is cleared.
    return pt_ma_quad(t, n_t, orb, k, k_per_band, ld, n_b, n_ss, t_exp, max_iter, y, wt, flux, ssr, scratch,
                      (size_t)PT_MA_NOALLOC_SCRATCH_BYTES, n_bad, stream);
}
