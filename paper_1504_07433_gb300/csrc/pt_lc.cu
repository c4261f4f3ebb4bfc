// pt_lc.cu -- light-curve kernels and their C ABI (include/pt.h).
//
// Kernels of the fused light-curve path (Secs. 2.1, 2.2, 3.2, 3.4):
//   setup_kernel        per geometry: conjunction anchor, double-float t0/P and
//                       a conservative transit window; per time: double-float split.
//   gim_window_kernel   window test of every (time, geometry) pair; the pairs in
//                       the window go to per-geometry lists, all others get flux 1
//                       (its leading CTAs also build the Gimenez tables).
//   gim_scan_kernel     work items of 128 listed pairs per geometry.
//   ma_pairs_kernel     Mandel-Agol: per item, the in-transit supersamples packed
//                       into one dense list, evaluated, summed per pair in
//                       supersample order, limb darkening per passband, stores.
//   gim_cheb_coef_kernel, gim_cheb_kernel
//                       Gimenez: the series in a Chebyshev basis (coefficients
//                       per geometry, then the evaluation over the dense lists).
//   gim_zi_table_kernel, gim_zi_kernel
//                       Gimenez interpolated in z (Sec. 3.3).
//   ma_lc_kernel        the tile kernel (256 times x 8 geometries per CTA) of the
//                       interpolated and allocation-free Mandel-Agol calls.
//   ssr_part_kernel / ssr_reduce_kernel
//                       residual sums in a fixed order.
// Every sum is formed in a fixed order, so results are bitwise reproducible.
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
constexpr int MAX_SS = 256;  // supersamples per exposure
constexpr int MAX_NEWTON = 64;  // cap on Newton steps
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
    int *cnt;            // per-geometry list counters to zero, or null
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
        if (g < s.n_geom) {
            make_geom(s, g, &s.rec[g]);
            if (s.cnt) s.cnt[g] = 0;
        }
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
    // interpolated Mandel-Agol terms (Sec. 2.2.3), when the kernel uses them
    const float4 *mtab;  // [n_k][n_z]: (lambda_e, lambda_d + 2/3 Theta, eta_d, 0)
    int mn_k, mn_z;
    float mk_lo, mk_hi, minv_dk, minv_dz;
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
        if (valid && pt::maybe_in_window(ts.x, srec[vl])) {
            dt = pt::reduce_time(ts.x, ts.y, srec[vl]);
            inw = (dt >= srec[vl].win_lo) && (dt <= srec[vl].win_hi);
        }
        sdt[vl][tl] = dt;
        sflag[vl][tl] = inw ? 1 : 0;
        if (__any_sync(0xffffffffu, inw)) {   // warp-uniform
            int slot = pt::warp_append(sqn, inw);
            if (inw) squeue[slot] = (unsigned short)(vl * TT + tl);
        }
    }
    __syncthreads();
}

__device__ __forceinline__ float ss_offset(float t_exp, int s, float inv_nss)
{
    return t_exp * (((float)s + 0.5f) * inv_nss - 0.5f);   // inv_nss = 1 / n_ss
}

// ---------------------------------------------------------------------------
// Mandel-Agol light curves
// ---------------------------------------------------------------------------
template <bool INTERP>
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
    const float inv_nss = 1.0f / (float)nss;

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
            float dts = sdt[vl][ti] + ss_offset(A.t_exp, s, inv_nss);
            bool bad = false;
            float z = pt::orbit_z<true>(r, dts, A.max_iter, &bad);
            if (bad) atomicAdd(&sbad, 1);
            if constexpr (INTERP)
                pt::ma_interp(A.mtab, A.mn_k, A.mn_z, A.mk_lo, A.mk_hi, A.minv_dk, A.minv_dz, r.k, z, &le, &ld, &ed);
            else
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
// Per geometry the table pass stores T_{n,j} = A_{n,j} G_j(nu+2, nu+1; 1-b)^2
// (Sec. 2.1.4: the z-independent factors).  Per (time, geometry) pair the
// evaluation accumulates, for n = 0..N,
//   alpha_n = b^2 (1 - c^2)^{nu+1} sum_j T_{n,j} G_j(nu+2, 1; c^2),
// with only summations and multiplications in the z-dependent part
// (Sec. 2.1.4).  Kernels:
//   gim_window_kernel  the tables (leading CTAs); then every pair: window
//                      test; pairs in the window go to a per-geometry list,
//                      the others get flux 1;
//   gim_scan_kernel    work items per geometry (ppi listed pairs each) and
//                      their exclusive prefix;
//   gim_cheb_coef_kernel / gim_cheb_kernel  the series in a Chebyshev basis
//                      shared by the orders (below): coefficients per
//                      geometry, then persistent CTAs that take work items
//                      from an atomic counter, evaluate the items' in-transit
//                      supersamples as a dense list and sum each pair's
//                      terms on the pair's own thread.
// Every pair's sums are taken in the same order whatever thread evaluated
// its terms and whatever CTA took its item, so the result is deterministic.
// ---------------------------------------------------------------------------
constexpr int GW_VT = 32;         // geometries per CTA of the window kernel (<= 32: one bit each)
constexpr int GS_THREADS = 128;   // threads per CTA of the evaluation kernels (one owned pair each)

struct GimArgs {
    const float2 *tsplit;
    int n_t;
    const GeomRec *rec;
    int n_geom;
    const float4 *gtab;   // [n_geom][N+1][n_j]: (r1_j, r2_j, r3_{j+1}, T_j)
    int N, n_j;
    const float *ld;      // [rows][N]
    int n_bpg;            // band rows per geometry
    int n_ss;
    float t_exp;
    int max_iter;
    float *flux;          // [rows][n_t]
    int *cnt;             // [n_geom] listed pairs per geometry
    int *pref;            // [n_geom + 1] work items before each position of the geometry order
    int *gord;            // [n_geom] geometry at each position of the order
    int *ctr;             // next work item of the evaluation kernel
    int *list;            // [n_geom][n_t] time indices of listed pairs
    int ppi;              // pairs per work item (GS_THREADS or MA_PPI)
    int *n_bad;
};

// Double-float arithmetic for the table recursion: a value is the unevaluated
// sum h + l of two floats (about 48 significant bits).  Sums and products
// carry their rounding errors exactly (Knuth's two-sum; the FMA form of
// Dekker's product).  GB300's FP64 rate is a small fraction of its FP32
// rate, so a chain of FP64 operations would dominate the table work.
struct DF {
    float h, l;
};

__device__ __forceinline__ DF df_of(double v)
{
    float h = (float)v;
    return DF{h, (float)(v - (double)h)};
}

__device__ __forceinline__ DF df_norm(float s, float e)   // |s| >= |e|
{
    float h = s + e;
    return DF{h, e - (h - s)};
}

__device__ __forceinline__ DF df_add(DF a, DF b)
{
    float s = a.h + b.h;
    float bb = s - a.h;
    float e = (a.h - (s - bb)) + (b.h - bb);
    return df_norm(s, e + (a.l + b.l));
}

__device__ __forceinline__ DF df_mul(DF a, DF b)
{
    float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
    return df_norm(p, e);
}

// a b + c with one two-sum: the product's rounding error (fmaf), the two-sum
// error of p + c_h, the cross terms and c_l go into the low part
__device__ __forceinline__ DF df_mad(DF a, DF b, DF c)
{
    const float p = a.h * b.h;
    const float e = fmaf(a.h, b.h, -p);
    const float s = p + c.h;
    const float bb = s - p;
    const float err = (p - (s - bb)) + (c.h - bb);
    return df_norm(s, fmaf(a.h, b.l, fmaf(a.l, b.h, c.l)) + (e + err));
}

// Gimenez per-geometry table for Clenshaw's summation: entry (n, j) packs the
// z-recursion coefficients r1_j, r2_j, r3_{j+1} of G_j(nu+2, 1; x) with
// T_{n,j} = A_{n,j} G_j(nu+2, nu+1; 1-b)^2, the z-independent factor of
// Sec. 2.1.4 (recursion in double-float arithmetic, stored FP32).
// A table CTA covers one order n and TABLE_GPC geometries (one thread each;
// the CTA's other threads only help stage row n of the plan's coefficients
// in shared memory as double-float pairs).  The recursion is a chain of n_j
// dependent steps per thread, so the chains are spread thinly over many SMs,
// and the table CTAs run inside the window kernel's launch, in the shadow of
// its wide grid.
constexpr int TABLE_GPC = 64;
struct TableJob {
    const float *k;           // [n_geom] radius ratio of each geometry (the call's k)
    int n_geom, NP1, n_j;
    const double *A, *recb;   // the plan's A_{n,j} and recursion of G_j(nu+2, nu+1; x), FP64
    const float4 *coef;       // the plan's recursion of G_j(nu+2, 1; x), FP32
    float4 *tab;              // [n_geom][NP1][n_j]
    int n_blocks;             // table CTAs (0: none)
};

__device__ __forceinline__ void table_cta(const TableJob &J, int n, int gb)
{
    extern __shared__ __align__(16) unsigned char tsm[];
    const int n_j = J.n_j;
    float4 *scf = reinterpret_cast<float4 *>(tsm);   // [n_j]
    DF *sA = reinterpret_cast<DF *>(scf + n_j);      // [n_j]
    DF *srb = sA + n_j;                              // [n_j][3]
    for (int i = threadIdx.x; i < n_j; i += blockDim.x) {
        scf[i] = J.coef[(size_t)n * n_j + i];
        sA[i] = df_of(J.A[(size_t)n * n_j + i]);
    }
    for (int i = threadIdx.x; i < 3 * n_j; i += blockDim.x) srb[i] = df_of(J.recb[(size_t)n * n_j * 3 + i]);
    __syncthreads();
    const int g = gb * TABLE_GPC + threadIdx.x;
    if (threadIdx.x >= TABLE_GPC || g >= J.n_geom) return;
    const double k = J.k[g];
    const DF x = df_of(1.0 - k / (1.0 + k));
    float4 *out = J.tab + ((size_t)g * J.NP1 + n) * n_j;
    DF gp = DF{0.0f, 0.0f}, gc = DF{1.0f, 0.0f};
    for (int j = 0; j < n_j; ++j) {
        float4 c = scf[j];
        float r3n = (j + 1 < n_j) ? scf[j + 1].z : 0.0f;
        DF t = df_mul(df_mul(sA[j], gc), gc);
        out[j] = make_float4(c.x, c.y, r3n, t.h + t.l);
        DF al = df_add(srb[3 * j], df_mul(srb[3 * j + 1], x));
        DF gn = df_add(df_mul(al, gc), df_mul(srb[3 * j + 2], gp));
        gp = gc;
        gc = gn;
    }
}

size_t gim_table_smem(int n_j) { return (size_t)n_j * (sizeof(float4) + 4 * sizeof(DF)); }

// The same table from the standalone launch (the Chebyshev path's side
// stream), with the chain threads doing only the recurrence: a chain runs
// alone on its scheduler, so its time is the length of its instruction
// stream.  Per CTA: order n, TABLE_GPC2 geometries.  All threads first form
// r1_j + r2_j x of every geometry and step, the chain threads (one per
// geometry) then run G_{j+1} = (r1 + r2 x) G_j + r3 G_{j-1} and keep each
// G_j, and all threads finally form T_{n,j} = A_{n,j} G_j^2 and store the
// packed rows.  The double-float operations are those of table_cta, so the
// table is bitwise the same.
constexpr int TABLE_GPC2 = 16;

size_t gim_table2_smem(int n_j)
{
    return (size_t)n_j * (sizeof(float4) + 4 * sizeof(DF)) + 2 * (size_t)TABLE_GPC2 * (n_j + 1) * sizeof(DF) +
           TABLE_GPC2 * sizeof(DF);
}

__device__ __forceinline__ void table_cta2(const TableJob &J, int n, int gb)
{
    extern __shared__ __align__(16) unsigned char tsm[];
    const int n_j = J.n_j;
    float4 *scf = reinterpret_cast<float4 *>(tsm);   // [n_j]
    DF *sA = reinterpret_cast<DF *>(scf + n_j);      // [n_j]
    DF *srb = sA + n_j;                              // [n_j][3]
    // rows of n_j + 1: the chain lanes, one geometry each, read and write
    // their rows at the same step without bank conflicts
    const int rs = n_j + 1;
    DF *sal = srb + 3 * n_j;                         // [TABLE_GPC2][n_j + 1]: r1_j + r2_j x
    DF *sG = sal + TABLE_GPC2 * rs;                  // [TABLE_GPC2][n_j + 1]: G_j
    DF *sx = sG + TABLE_GPC2 * rs;                   // [TABLE_GPC2]: x = 1 - b
    const int tid = threadIdx.x;
    const int g0 = gb * TABLE_GPC2;
    const int ng = min(TABLE_GPC2, J.n_geom - g0);
    for (int i = tid; i < n_j; i += blockDim.x) {
        scf[i] = J.coef[(size_t)n * n_j + i];
        sA[i] = df_of(J.A[(size_t)n * n_j + i]);
    }
    for (int i = tid; i < 3 * n_j; i += blockDim.x) srb[i] = df_of(J.recb[(size_t)n * n_j * 3 + i]);
    if (tid < ng) {
        const double k = J.k[g0 + tid];
        sx[tid] = df_of(1.0 - k / (1.0 + k));
    }
    __syncthreads();
    for (int j = tid; j < n_j; j += blockDim.x)
        for (int gl = 0; gl < ng; ++gl) sal[gl * rs + j] = df_add(srb[3 * j], df_mul(srb[3 * j + 1], sx[gl]));
    __syncthreads();
    if (tid < ng) {
        const DF *al = sal + tid * rs;
        DF *G = sG + tid * rs;
        // G_{j+1} = al_j G_j + r3_j G_{j-1}; q = r3_j G_{j-1} is formed one
        // step ahead, so each step's dependent path is one df_mad
        DF gc = DF{1.0f, 0.0f}, q = DF{0.0f, 0.0f};
        for (int j = 0; j < n_j; ++j) {
            G[j] = gc;
            const DF gn = df_mad(al[j], gc, q);
            if (j + 1 < n_j) q = df_mul(srb[3 * (j + 1) + 2], gc);
            gc = gn;
        }
    }
    __syncthreads();
    for (int j = tid; j < n_j; j += blockDim.x) {
        const float4 c = scf[j];
        const float r3n = (j + 1 < n_j) ? scf[j + 1].z : 0.0f;
        for (int gl = 0; gl < ng; ++gl) {
            const DF gc = sG[gl * rs + j];
            const DF t = df_mul(df_mul(sA[j], gc), gc);
            J.tab[((size_t)(g0 + gl) * J.NP1 + n) * n_j + j] = make_float4(c.x, c.y, r3n, t.h + t.l);
        }
    }
}

// One CTA covers TT times x GW_VT geometries.  The first pass of the window
// test (as pt::maybe_in_window, but with its margin bounded once per tile and
// geometry from the tile's largest |t_h|) costs a subtraction, a product, a
// rounding, an FMA and two comparisons per pair against constants staged in
// shared memory; candidates then take the exact double-float test.  Appends
// in two passes over a per-thread bit mask: ballots count each warp's pairs
// per geometry, one global atomic per geometry reserves the CTA's stretch of
// its list, and the same ballots place every pair (warp order, then lane
// order) inside that stretch.  Every other pair gets flux 1.
__device__ __forceinline__ void window_cta(const GimArgs &A, int bx, int by)
{
    constexpr int NW = TT / 32;
    __shared__ GeomRec srec[GW_VT];
    __shared__ float4 stest[GW_VT];   // t0_h, 1/P, P_h, win_lo - m
    __shared__ float shi[GW_VT];      // win_hi + m
    __shared__ int swc[NW][GW_VT];    // pairs per (warp, geometry), then the warp's offset
    __shared__ int sbase[GW_VT];
    __shared__ float swmax[NW];
    const int tl = threadIdx.x, lane = tl & 31, warp = tl >> 5;
    const int g0 = by * GW_VT;
    const int ng = min(GW_VT, A.n_geom - g0);
    for (int i = tl; i < ng * 6; i += TT) {
        int vl = i / 6, c = i % 6;
        reinterpret_cast<float4 *>(&srec[vl])[c] = reinterpret_cast<const float4 *>(&A.rec[g0 + vl])[c];
    }
    const int t = bx * TT + tl;
    const bool tv = t < A.n_t;
    const float2 ts = tv ? A.tsplit[t] : make_float2(0.0f, 0.0f);
    // the tile's largest |t_h| (non-negative floats order like their bits)
    float am = __int_as_float(__reduce_max_sync(0xffffffffu, __float_as_int(fabsf(ts.x))));
    if (lane == 0) swmax[warp] = am;
    __syncthreads();
    if (tl < ng) {
        float tmax = swmax[0];
        for (int w = 1; w < NW; ++w) tmax = fmaxf(tmax, swmax[w]);
        const GeomRec &r = srec[tl];
        // the margin of pt::maybe_in_window with |s| <= |t_h| + |t0_h|,
        // |n| P_h <= |s| + P_h / 2 and |d| <= P_h / 2
        float m = 1.2e-7f * (3.0f * tmax + 3.0f * fabsf(r.t0h) + r.Ph) + 1e-9f;
        stest[tl] = make_float4(r.t0h, r.invP, r.Ph, r.win_lo - m);
        shi[tl] = r.win_hi + m;
    }
    __syncthreads();
    unsigned bits = 0u;
    if (tv) {
        const float th = ts.x;
        // first pass without branches: a mask of the candidates ...
        unsigned cand = 0u;
#pragma unroll 8
        for (int vl = 0; vl < ng; ++vl) {
            const float4 q = stest[vl];
            const float sv = th - q.x;
            const float d = fmaf(-rintf(sv * q.y), q.z, sv);
            cand |= ((d >= q.w) & (d <= shi[vl])) ? (1u << vl) : 0u;
        }
        // ... then the exact test for those only
        for (unsigned rest = cand; rest; rest &= rest - 1u) {
            const int vl = __ffs(rest) - 1;
            const float dt = pt::reduce_time(th, ts.y, srec[vl]);
            if ((dt >= srec[vl].win_lo) && (dt <= srec[vl].win_hi)) bits |= 1u << vl;
        }
    }
    // geometries with a pair in this warp (the ballots below visit only those)
    const unsigned wbits = __reduce_or_sync(0xffffffffu, bits);
    if (lane < GW_VT) swc[warp][lane] = 0;
    __syncwarp();
    for (unsigned rest = wbits; rest; rest &= rest - 1u) {
        const int vl = __ffs(rest) - 1;
        unsigned mb = __ballot_sync(0xffffffffu, (bits >> vl) & 1u);
        if (lane == 0) swc[warp][vl] = __popc(mb);
    }
    __syncthreads();
    if (tl < ng) {   // per geometry: warp offsets, then one reservation
        int run = 0;
        for (int w = 0; w < NW; ++w) {
            int c = swc[w][tl];
            swc[w][tl] = run;
            run += c;
        }
        sbase[tl] = run > 0 ? atomicAdd(A.cnt + g0 + tl, run) : 0;
    }
    __syncthreads();
    {
        const unsigned lt = (1u << lane) - 1u;
        for (unsigned rest = wbits; rest; rest &= rest - 1u) {
            const int vl = __ffs(rest) - 1;
            const bool in = (bits >> vl) & 1u;
            unsigned mb = __ballot_sync(0xffffffffu, in);
            if (in) A.list[(size_t)(g0 + vl) * A.n_t + sbase[vl] + swc[warp][vl] + __popc(mb & lt)] = t;
        }
    }
    if (tv) {
        const size_t row_stride = (size_t)A.n_t;
        float *fp = A.flux + (size_t)g0 * A.n_bpg * row_stride + t;
        if (A.n_bpg == 1) {
#pragma unroll 8
            for (int vl = 0; vl < ng; ++vl, fp += row_stride)
                if (!((bits >> vl) & 1u)) *fp = 1.0f;
        } else {
            for (int vl = 0; vl < ng; ++vl)
                for (int bb = 0; bb < A.n_bpg; ++bb, fp += row_stride)
                    if (!((bits >> vl) & 1u)) *fp = 1.0f;
        }
    }
}

// One launch: J.n_blocks table CTAs first (they start first and run in the
// shadow of the window CTAs), then n_tiles x ceil(n_geom / GW_VT) window CTAs.
__global__ void __launch_bounds__(TT) gim_window_kernel(GimArgs A, TableJob J, int n_tiles)
{
    int id = blockIdx.x;
    if (id < J.n_blocks) {
        table_cta(J, id % J.NP1, id / J.NP1);
        return;
    }
    id -= J.n_blocks;
    window_cta(A, id % n_tiles, id / n_tiles);
}

// The table alone (table_cta2): the Chebyshev path launches it on the plan's
// side stream at the start of the call (it needs only k), beside the set-up
// and window kernels.
__global__ void __launch_bounds__(TT) gim_table_kernel(TableJob J)
{
    table_cta2(J, blockIdx.x % J.NP1, blockIdx.x / J.NP1);
}

// pref[g] = sum over g' < g of ceil(cnt[g'] / ppi); pref[n_geom] = total.
// One CTA of 1024 threads; also rewinds the evaluation kernels' item counter.
// Work items in a cost order: geometries sorted by an estimate of the
// in-transit supersamples per listed pair, largest first, so that the items
// handed out last are the cheap ones and the persistent CTAs finish close
// together.  The window of a geometry is its transit plus half an exposure on
// each side (and margins), so a listed pair is in transit for about a
// fraction (W - t_exp) / W of its exposure, W = win_hi - win_lo.  Ties (and
// every geometry when there is no exposure time) keep their index order.
// gord[p] is the geometry at position p; pref[p] the items before position p.
// Up to 1,024 geometries each thread counts the geometries before its own
// (no barriers), up to SCAN_SORT_MAX a bitonic sort in shared memory, above
// that the order is the index order.  The Mandel-Agol pairs kernel (order =
// false: items of a few microseconds, and measured slower with the cost
// order) takes the index order.
constexpr int SCAN_SORT_MAX = 4096;

__device__ __forceinline__ float scan_key(const int *cnt, const GeomRec *rec, float t_exp, int g)
{
    const float w = rec[g].win_hi - rec[g].win_lo;
    return (cnt[g] > 0 && w > 0.0f) ? fmaxf(w - t_exp, 0.0f) / w : -1.0f;
}

__global__ void __launch_bounds__(1024) gim_scan_kernel(const int *cnt, const GeomRec *rec, float t_exp, int n_geom,
                                                        int ppi, bool order, int *pref, int *gord, int *ctr)
{
    __shared__ int swarp[32];
    __shared__ int scarry;
    __shared__ float skey[SCAN_SORT_MAX];
    __shared__ int sidx[SCAN_SORT_MAX];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarp = blockDim.x >> 5;
    const bool sorted = order && n_geom <= SCAN_SORT_MAX;
    if (threadIdx.x == 0) {
        scarry = 0;
        *ctr = 0;
    }
    if (sorted && n_geom <= (int)blockDim.x) {
        // one thread per geometry: its position is the number of geometries
        // before it in the order
        const int i = threadIdx.x;
        if (i < n_geom) skey[i] = scan_key(cnt, rec, t_exp, i);
        __syncthreads();
        if (i < n_geom) {
            const float ki = skey[i];
            int r = 0;
            for (int j = 0; j < n_geom; ++j) {
                const float kj = skey[j];
                r += (kj > ki || (kj == ki && j < i)) ? 1 : 0;
            }
            sidx[r] = i;
        }
        __syncthreads();
    } else if (sorted) {
        int n2 = 1;
        while (n2 < n_geom) n2 <<= 1;
        for (int i = threadIdx.x; i < n2; i += blockDim.x) {
            skey[i] = i < n_geom ? scan_key(cnt, rec, t_exp, i) : -2.0f;   // padding sorts last
            sidx[i] = i;
        }
        __syncthreads();
        // bitonic sort: key descending, index ascending among equal keys
        for (int kk = 2; kk <= n2; kk <<= 1) {
            for (int j = kk >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                    const int l = i ^ j;
                    if (l > i) {
                        const float ki = skey[i], kl = skey[l];
                        const int ii = sidx[i], il = sidx[l];
                        const bool i_first = ki > kl || (ki == kl && ii < il);
                        const bool up = (i & kk) == 0;   // this block in the final order
                        if (up != i_first) {
                            skey[i] = kl;
                            skey[l] = ki;
                            sidx[i] = il;
                            sidx[l] = ii;
                        }
                    }
                }
                __syncthreads();
            }
        }
    }
    for (int p = threadIdx.x; p < n_geom; p += blockDim.x) gord[p] = sorted ? sidx[p] : p;
    __syncthreads();
    for (int base = 0; base < n_geom; base += blockDim.x) {
        int p = base + threadIdx.x;
        int v = (p < n_geom) ? (cnt[sorted ? sidx[p] : p] + ppi - 1) / ppi : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) swarp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = (lane < nwarp) ? swarp[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            swarp[lane] = w;
        }
        __syncthreads();
        int incl = scarry + (warp > 0 ? swarp[warp - 1] : 0) + x;
        if (p < n_geom) pref[p] = incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) scarry = incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) pref[n_geom] = scarry;
}

// ---------------------------------------------------------------------------
// Chebyshev form of the series.  For one geometry and order n,
//   S_n(x) = sum_{j < n_j} T_{n,j} G_j(nu+2, 1; x)
// is a polynomial of degree n_j - 1 in x, so it has an exact expansion
//   S_n(x) = sum_{m < n_j} d_{n,m} T_m(y),   y = 2x - 1.
// The Chebyshev basis does not depend on n, so one recurrence
// T_{m+1} = 2y T_m - T_{m-1} per supersample serves all N + 1 orders:
// N + 2 FMAs per term instead of 3 (N + 1).
// gim_cheb_coef_kernel forms the d_{n,m} by Clenshaw's backward summation of
// the Jacobi series (the recursion of Sec. 2.1.4, the table's r1_j, r2_j,
// r3_{j+1}, T_{n,j}),
//   b_j = T_j + (r1_j + r2_j x) b_{j+1} + r3_{j+1} b_{j+2},   S_n = b_0,
// carried out on Chebyshev coefficient vectors instead of values: with
// x = (1 + y)/2, multiplying by x is (1/2)(b + y b), and y T_m =
// (T_{m+1} + T_{m-1})/2 (y T_0 = T_1), so (y b)_m = (b_{m-1} + b_{m+1})/2,
// (y b)_0 = b_1 / 2, (y b)_1 = b_0 + b_2 / 2.  Each step touches every
// coefficient once (about n_j^2 / 2 x 3 FMAs per order in all); in FP32 the
// alpha_n it leads to stay within ~1e-7 of the FP64 series (emulated at
// n_j = 192 over k = 0.05 .. 0.2), the level of the FP32 evaluation.
// One warp per (geometry, order): lane l holds coefficients l S .. l S + S - 1
// in registers, so a step needs the two neighbours across lanes only (two
// shuffles); the table row sits in the warp's shared memory, read by
// broadcast.  Warps for the row padding (orders N + 1 .. DS - 1) write zeros.
// ---------------------------------------------------------------------------
constexpr int CW_WARPS = 1;   // warps per CTA of the coefficient kernel (one: the scheduler spreads the chains evenly)

template <int S>
__global__ void __launch_bounds__(32 * CW_WARPS) gim_cheb_coef_kernel(const float4 *gtab, int NP1, int n_j, int DS,
                                                                     float *dtab)
{
    extern __shared__ __align__(16) float4 ctab_sm[];   // [CW_WARPS][n_j]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x;
    const int n = blockIdx.y * CW_WARPS + warp;
    if (n >= DS) return;   // a whole warp; the kernel has no CTA-wide barrier
    float *out = dtab + (size_t)g * n_j * DS + n;   // d_{n,m} at out[m DS]
    if (n >= NP1) {
        for (int m = lane; m < n_j; m += 32) out[(size_t)m * DS] = 0.0f;
        return;
    }
    float4 *tab = ctab_sm + warp * n_j;
    const float4 *src = gtab + ((size_t)g * NP1 + n) * n_j;
    for (int j = lane; j < n_j; j += 32) tab[j] = src[j];
    __syncwarp();
    float b1[S], b2[S];
    float wl[S];   // weight of the lower neighbour in (y b)_m: 1/2, 1 at m = 1, 0 at m = 0
    const int m0 = lane * S;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        b1[s] = b2[s] = 0.0f;
        wl[s] = (m0 + s == 0) ? 0.0f : (m0 + s == 1 ? 1.0f : 0.5f);
    }
    // one step: from (bn = b_{j+1}, bo = b_{j+2}) to b_j, written over bo
    auto step = [&](int j, float (&bn)[S], float (&bo)[S]) {
        const float4 c = tab[j];
        const float a = fmaf(0.5f, c.y, c.x);   // the part of r1 + r2 x without y
        const float h = 0.5f * c.y;             // the coefficient of y b
        const float left = __shfl_up_sync(0xffffffffu, bn[S - 1], 1);   // b_{m0 - 1}
        const float right = __shfl_down_sync(0xffffffffu, bn[0], 1);   // b_{m0 + S}
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const float bl = (s == 0) ? left : bn[s - 1];
            const float br = (s == S - 1) ? (lane == 31 ? 0.0f : right) : bn[s + 1];
            const float yb = fmaf(wl[s], bl, 0.5f * br);
            bo[s] = fmaf(a, bn[s], fmaf(h, yb, c.z * bo[s]));
        }
        if (lane == 0) bo[0] += c.w;             // + T_j (degree 0)
    };
    int j = n_j - 1;
#pragma unroll 1
    for (; j >= 1; j -= 2) {
        step(j, b1, b2);       // b_j into b2
        step(j - 1, b2, b1);   // b_{j-1} into b1
    }
    if (j == 0) {
        step(0, b1, b2);
#pragma unroll
        for (int s = 0; s < S; ++s) b1[s] = b2[s];
    }
#pragma unroll
    for (int s = 0; s < S; ++s)
        if (m0 + s < n_j) out[(size_t)(m0 + s) * DS] = b1[s];
}

// coefficients per lane of the coefficient kernel for a series depth
int gim_cheb_coef_s(int n_j) { return (n_j + 31) / 32; }

// Evaluation over the pair lists.  Persistent CTAs take items of GS_THREADS
// listed pairs of one geometry and stage its coefficient rows once per item.
// An item runs in batches of up to GS_SSB supersamples:
//  1. each thread (one pair) computes z at the batch's supersamples and keeps
//     the in-transit ones, (y = 2x - 1, q = sqrt(1 - x)) with x = c^2, in
//     order; a scan over the CTA places every pair's entries in one dense
//     list (pair-major, supersample-minor);
//  2. the list is cut into rounds; in a round each thread evaluates G
//     consecutive entries, whatever pairs they belong to, so that no lane
//     idles on an out-of-transit supersample: one Chebyshev recurrence per
//     entry, T_{m+1} = 2y T_m - T_{m-1}, and one FMA per order n and m for
//     d_{n,m} T_m, two orders per two-lane FMA instruction (fma.rn.f32x2:
//     a third fewer instructions than scalar FMAs, and measured on this
//     part 0.68 of the FP32 peak in series multiply-adds against 0.52 for
//     the scalar form of the same loop).  Rounds of GS_GMAX = 4 entries per
//     thread while at least 4 GS_THREADS entries are left, then one round of
//     the fewest entries per thread (1 to 3) that holds the rest (each
//     coefficient load serves the thread's entries).  The S_n go to shared
//     memory;
//  3. each thread adds its own pair's b^2 q^(n+4) S_n to alpha_n in
//     supersample order, so the sums do not depend on the rounds.
// After the last batch, the passband combination of Sec. 2.1.3.
constexpr int GS_SSB = 16;    // supersamples per batch of the Chebyshev kernel
constexpr int GS_GMAX = 4;    // entries per thread in the largest round
constexpr int GS_WROWS = 8;   // passbands whose combination weights are staged per geometry

// The geometry of work item it: the largest g with pref[g] <= it (pref is
// non-decreasing, pref[0] = 0 <= it), found by one warp: each round splits
// [lo, hi] into 32 strides and loads their first entries in parallel, the
// lanes whose entry is <= it form a prefix, and its last lane brackets the
// answer.  Two rounds (two dependent loads) up to 1,024 geometries.
__device__ __forceinline__ int item_geometry(const int *pref, int n_geom, int it, int lane)
{
    int lo = 0, hi = n_geom - 1;
    for (;;) {
        const int step = (hi - lo + 32) / 32;   // ceil((hi - lo + 1) / 32)
        const int idx = lo + lane * step;
        const bool ok = idx <= hi && pref[idx] <= it;
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        lo += (31 - __clz(m)) * step;
        if (step == 1) return lo;
        hi = min(hi, lo + step - 1);
    }
}

// (a0, a1) += (d0, d1) w as one two-lane FMA (sm_100 and later).  Each lane
// is a fused multiply-add rounded once, so the result is that of two fmaf.
__device__ __forceinline__ void fma2_pair(float d0, float d1, float w, float &a0, float &a1)
{
    float2 a = make_float2(a0, a1);
    const float2 d = make_float2(d0, d1);
    const float2 ww = make_float2(w, w);
    asm("fma.rn.f32x2 %0, %1, %2, %0;"
        : "+l"(*reinterpret_cast<unsigned long long *>(&a))
        : "l"(*reinterpret_cast<const unsigned long long *>(&d)), "l"(*reinterpret_cast<const unsigned long long *>(&ww)));
    a0 = a.x;
    a1 = a.y;
}

template <int NP1, int G>
__device__ __forceinline__ void cheb_eval(const float *sd, int nj, const float (&y)[G], float (&acc)[G][NP1])
{
    constexpr int DS = (NP1 + 3) & ~3;
    float wa[G], wb[G], a2[G];
#pragma unroll
    for (int e = 0; e < G; ++e) {
        a2[e] = y[e] + y[e];
        wa[e] = 1.0f;
        wb[e] = y[e];
#pragma unroll
        for (int n = 0; n < NP1; ++n) acc[e][n] = fmaf(sd[DS + n], wb[e], sd[n]);
    }
    // one step: T_m = 2y T_{m-1} - T_{m-2} in place of T_{m-2} (wa for even m,
    // wb for odd m, so the loop carries no register copies)
    auto step = [&](int m, float (&wn)[G], const float (&wp)[G]) {
        float dm[DS];
        const float4 *row = reinterpret_cast<const float4 *>(sd + m * DS);
#pragma unroll
        for (int n = 0; n < DS; n += 4) {
            const float4 v = row[n / 4];
            dm[n] = v.x;
            dm[n + 1] = v.y;
            dm[n + 2] = v.z;
            dm[n + 3] = v.w;
        }
#pragma unroll
        for (int e = 0; e < G; ++e) {
            wn[e] = fmaf(a2[e], wp[e], -wn[e]);
            // orders in pairs through the two-lane FMA (each lane one FMA,
            // rounded once: the same result as two fmaf), the odd last order
            // scalar
#pragma unroll
            for (int n = 0; n + 1 < NP1; n += 2) fma2_pair(dm[n], dm[n + 1], wn[e], acc[e][n], acc[e][n + 1]);
            if (NP1 & 1) acc[e][NP1 - 1] = fmaf(dm[NP1 - 1], wn[e], acc[e][NP1 - 1]);
        }
    };
    int m = 2;
#pragma unroll 2
    for (; m + 1 < nj; m += 2) {
        step(m, wa, wb);
        step(m + 1, wb, wa);
    }
    if (m < nj) step(m, wa, wb);
}

// One round: entries [r0, r0 + G GS_THREADS) of the dense list (those below
// n_e), G consecutive ones per thread; S_n to sS[n][slot].
template <int NP1, int G>
__device__ __forceinline__ void cheb_round(const float *sd, int nj, const float2 *syq, const int *sst, float *sS,
                                           int r0, int n_e)
{
    constexpr int CH = GS_GMAX * GS_THREADS;
    const int tid = threadIdx.x;
    const int e0 = r0 + G * tid;
    if (e0 >= n_e) return;
    float y[G];
    int p = 0;
    {
        int lo = 0, hi = GS_THREADS - 1;   // the last pair with sst[p] <= e0
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sst[mid] <= e0) lo = mid;
            else hi = mid - 1;
        }
        p = lo;
    }
#pragma unroll
    for (int u = 0; u < G; ++u) {
        const int e = e0 + u;
        y[u] = 0.0f;
        if (e < n_e) {
            while (sst[p + 1] <= e) ++p;
            y[u] = syq[(e - sst[p]) * GS_THREADS + p].x;
        }
    }
    float acc[G][NP1];
    cheb_eval<NP1, G>(sd, nj, y, acc);
#pragma unroll
    for (int n = 0; n < NP1; ++n) {
        float *dst = sS + n * CH + G * tid;
        if (G % 4 == 0) {
#pragma unroll
            for (int u = 0; u < G; u += 4)
                *reinterpret_cast<float4 *>(dst + u) = make_float4(acc[u][n], acc[u + 1][n], acc[u + 2][n], acc[u + 3][n]);
        } else if (G % 2 == 0) {
#pragma unroll
            for (int u = 0; u < G; u += 2) *reinterpret_cast<float2 *>(dst + u) = make_float2(acc[u][n], acc[u + 1][n]);
        } else {
#pragma unroll
            for (int u = 0; u < G; ++u) dst[u] = acc[u][n];
        }
    }
}

template <int NP1>
__global__ void __launch_bounds__(GS_THREADS, 5) gim_cheb_kernel(GimArgs A, const float *dtab)
{
    constexpr int DS = (NP1 + 3) & ~3;        // floats per coefficient row
    constexpr int CH = GS_GMAX * GS_THREADS;  // entries of the largest round
    const int nj = A.n_j;
    const int nss = A.n_ss;
    const int ssb = min(nss, GS_SSB);
    extern __shared__ __align__(16) unsigned char dsm[];
    float *sd = reinterpret_cast<float *>(dsm);                  // [n_j][DS] coefficient rows
    float *sS = sd + nj * DS;                                    // [NP1][CH] series values of a round
    float2 *syq = reinterpret_cast<float2 *>(sS + NP1 * CH);     // [ssb][GS_THREADS] (y, q) per pair
    __shared__ GeomRec srec;
    __shared__ int sitem, sgeom, sfirst, scount, sbad;
    __shared__ float swt[GS_WROWS][NP1 + 1];   // per passband: 1 - sum u, u_1..u_N, D
    __shared__ int sst[GS_THREADS + 1];   // first dense entry of each pair; sst[GS_THREADS] = entries
    __shared__ int swarp[GS_THREADS / 32];
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int total = A.pref[A.n_geom];
    const float inv_nss = 1.0f / (float)nss;
    int nbad = 0;
    int staged = -1;
    if (tid == 0) sbad = 0;
#pragma unroll 1
    for (;;) {
        if (warp == 0) {
            int it = 0;
            if (lane == 0) it = atomicAdd(A.ctr, 1);
            it = __shfl_sync(0xffffffffu, it, 0);
            if (it < total) {
                const int pos = item_geometry(A.pref, A.n_geom, it, lane);
                if (lane == 0) {
                    const int g = A.gord[pos];
                    sgeom = g;
                    sfirst = A.pref[pos];
                    scount = A.cnt[g];
                }
            }
            if (lane == 0) sitem = it;
        }
        __syncthreads();
        const int it = sitem;
        const int g = sgeom;
        if (it >= total) break;   // uniform over the CTA
        if (g != staged) {
            const float4 *src = reinterpret_cast<const float4 *>(dtab + (size_t)g * nj * DS);
            float4 *dst = reinterpret_cast<float4 *>(sd);
            for (int i = tid; i < nj * DS / 4; i += GS_THREADS) dst[i] = src[i];
            if (tid < 6) reinterpret_cast<float4 *>(&srec)[tid] = reinterpret_cast<const float4 *>(&A.rec[g])[tid];
            if (tid < A.n_bpg && tid < GS_WROWS) {
                // C_0 D = 1 - sum u, C_n D = u_n, D = 1 - sum n u_n/(n+2)   (Sec. 2.1.3)
                const float *u = A.ld + ((size_t)g * A.n_bpg + tid) * A.N;
                float su = 0.0f, sdn = 0.0f;
#pragma unroll
                for (int n = 1; n < NP1; ++n) {
                    const float un = u[n - 1];
                    su += un;
                    sdn += (float)n * un / (float)(n + 2);
                    swt[tid][n] = un;
                }
                swt[tid][0] = 1.0f - su;
                swt[tid][NP1] = 1.0f - sdn;
            }
            staged = g;
        }
        __syncthreads();
        const int i = (it - sfirst) * GS_THREADS + tid;
        const bool own = i < scount;
        const int t = own ? A.list[(size_t)g * A.n_t + i] : 0;
        float dt = 0.0f;
        if (own) {
            const float2 ts = A.tsplit[t];
            dt = pt::reduce_time(ts.x, ts.y, srec);
        }
        const float kk = srec.k;
        const float bk = kk / (1.0f + kk);
        const float b2 = bk * bk;
        float al[NP1];   // alpha sums over the supersamples
#pragma unroll
        for (int n = 0; n < NP1; ++n) al[n] = 0.0f;
        float warm[3] = {__int_as_float(0x7fffffff), 0.0f, 0.0f};   // Kepler warm start (none yet)
#pragma unroll 1
        for (int sb0 = 0; sb0 < nss; sb0 += ssb) {
            // 1. in-transit supersamples of this pair, in order
            int c = 0;
            if (own) {
                const int s1 = min(nss, sb0 + ssb);
#pragma unroll 1
                for (int s = sb0; s < s1; ++s) {
                    bool bad = false;
                    const float z = pt::orbit_z<true, true>(srec, dt + ss_offset(A.t_exp, s, inv_nss), A.max_iter, &bad, warm);
                    if (bad) ++nbad;
                    if (z < 1.0f + kk) {
                        // z < 1 + k; the rounded reciprocal may put cz an ulp above 1
                        const float cz = fminf(z * pt::rcp_a(1.0f + kk), 1.0f);
                        const float x = cz * cz;
                        // (1 - cz)(1 + cz) is 0 or at least ~2^-24: a normal argument
                        syq[c * GS_THREADS + tid] = make_float2(fmaf(2.0f, x, -1.0f), pt::sqrt_a((1.0f - cz) * (1.0f + cz)));
                        ++c;
                    }
                }
            }
            // exclusive scan of the counts over the CTA
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane == 31) swarp[warp] = incl;
            __syncthreads();
            int base = 0;
#pragma unroll
            for (int w = 0; w < GS_THREADS / 32; ++w) base += (w < warp) ? swarp[w] : 0;
            sst[tid] = base + incl - c;
            if (tid == GS_THREADS - 1) sst[GS_THREADS] = base + incl;
            __syncthreads();
            const int n_e = sst[GS_THREADS];
            const int my0 = sst[tid];
            int r0 = 0;
#pragma unroll 1
            while (r0 < n_e) {
                // 2. a round of series values; its size from what is left
                const int rem = n_e - r0;
                int size;
                const int gfit = (rem + GS_THREADS - 1) / GS_THREADS;   // the last round fits what is left
                if (gfit >= GS_GMAX) {
                    cheb_round<NP1, GS_GMAX>(sd, nj, syq, sst, sS, r0, n_e);
                    size = GS_GMAX * GS_THREADS;
                } else if (gfit == 3) {
                    cheb_round<NP1, 3>(sd, nj, syq, sst, sS, r0, n_e);
                    size = 3 * GS_THREADS;
                } else if (gfit == 2) {
                    cheb_round<NP1, 2>(sd, nj, syq, sst, sS, r0, n_e);
                    size = 2 * GS_THREADS;
                } else {
                    cheb_round<NP1, 1>(sd, nj, syq, sst, sS, r0, n_e);
                    size = GS_THREADS;
                }
                __syncthreads();
                // 3. this pair's entries of the round, in supersample order:
                //    alpha_n += b^2 q^(n+4) S_n
                const int ea = max(my0, r0), eb = min(my0 + c, r0 + size);
#pragma unroll 1
                for (int e = ea; e < eb; ++e) {
                    const float qu = syq[(e - my0) * GS_THREADS + tid].y;
                    const float qq = qu * qu;
                    float w = b2 * qq * qq;
#pragma unroll
                    for (int n = 0; n < NP1; n += 2) {
                        al[n] = fmaf(sS[n * CH + (e - r0)], w, al[n]);
                        if (n + 1 < NP1) al[n + 1] = fmaf(sS[(n + 1) * CH + (e - r0)], w * qu, al[n + 1]);
                        w *= qq;
                    }
                }
                __syncthreads();
                r0 += size;
            }
        }
        if (own) {
#pragma unroll 1
            for (int bb = 0; bb < A.n_bpg; ++bb) {
                size_t row = (size_t)g * A.n_bpg + bb;
                // C_0 = (1 - sum u)/D, C_n = u_n/D, D = 1 - sum n u_n/(n+2)   (Sec. 2.1.3);
                // the first GS_WROWS passbands' (1 - sum u, u_n, D) were staged
                // with the geometry, the others are formed here the same way
                float wt[NP1 + 1];
                if (bb < GS_WROWS) {
#pragma unroll
                    for (int n = 0; n <= NP1; ++n) wt[n] = swt[bb][n];
                } else {
                    const float *u = A.ld + row * A.N;
                    float su = 0.0f, sdn = 0.0f;
#pragma unroll
                    for (int n = 1; n < NP1; ++n) {
                        const float un = u[n - 1];
                        su += un;
                        sdn += (float)n * un / (float)(n + 2);
                        wt[n] = un;
                    }
                    wt[0] = 1.0f - su;
                    wt[NP1] = 1.0f - sdn;
                }
                float acc_f = wt[0] * al[0];
#pragma unroll
                for (int n = 1; n < NP1; ++n) acc_f = fmaf(wt[n], al[n], acc_f);
                A.flux[row * A.n_t + t] = 1.0f - acc_f / wt[NP1] * inv_nss;
            }
        }
    }
    if (nbad) atomicAdd(&sbad, nbad);
    __syncthreads();
    if (tid == 0 && sbad && A.n_bad) atomicAdd(A.n_bad, sbad);
}

// floats per coefficient row: the N + 1 orders, padded to 16 bytes
int gim_cheb_ds(int N) { return (N + 4) & ~3; }
// coefficient rows, a round of series values and a batch of (y, q) entries
size_t gim_cheb_smem(int n_j, int N, int n_ss)
{
    return ((size_t)n_j * gim_cheb_ds(N) + (size_t)(N + 1) * GS_GMAX * GS_THREADS) * sizeof(float) +
           (size_t)GS_THREADS * (n_ss < GS_SSB ? n_ss : GS_SSB) * sizeof(float2);
}

// ---------------------------------------------------------------------------
// Gimenez model interpolated in z (Sec. 3.3).  gim_zi_table_kernel evaluates
// alpha_0..alpha_N of every geometry on its z nodes (n_in over [0, zb],
// zb = max(1 - k, 0), then n_edge over (zb, 1 + k]) with the same Clenshaw
// summation as the coefficient kernel's node values; gim_zi_kernel reads
// them by linear interpolation for every listed (time, geometry) pair (one
// thread per pair), with the same work items and passband combination as
// the series evaluation.
// ---------------------------------------------------------------------------
constexpr int ZI_MAX_VALUES = 16384;   // (n_in + n_edge)(N + 1) per geometry

struct ZiGrid {
    float zb, h1, h2, inv_h1, inv_h2;
};

__device__ __forceinline__ ZiGrid zi_grid(float k, int n_in, int n_edge)
{
    ZiGrid q;
    q.zb = fmaxf(1.0f - k, 0.0f);
    q.h1 = q.zb / (float)(n_in - 1);
    q.h2 = (1.0f + k - q.zb) / (float)n_edge;
    q.inv_h1 = (q.zb > 0.0f) ? 1.0f / q.h1 : 0.0f;
    q.inv_h2 = 1.0f / q.h2;
    return q;
}

__global__ void __launch_bounds__(128) gim_zi_table_kernel(const GeomRec *rec, const float4 *gtab, int NP1, int n_j,
                                                          int n_in, int n_edge, float *atab)
{
    const int g = blockIdx.x;
    const int nz = n_in + n_edge;
    const float kk = rec[g].k;
    const ZiGrid G = zi_grid(kk, n_in, n_edge);
    const float4 *tab = gtab + (size_t)g * NP1 * n_j;
    const float bk = kk / (1.0f + kk);
    const float b2 = bk * bk;
    for (int i = threadIdx.x; i < nz; i += blockDim.x) {
        float z = (i < n_in) ? (float)i * G.h1 : G.zb + (float)(i - n_in + 1) * G.h2;
        float x = 0.0f, q = 0.0f;
        if (z < 1.0f + kk) {
            float c = z / (1.0f + kk);
            x = c * c;
            q = sqrtf((1.0f - c) * (1.0f + c));
        }
        float *out = atab + ((size_t)g * nz + i) * NP1;
        for (int n = 0; n < NP1; ++n) {
            const float4 *tn = tab + (size_t)n * n_j;
            float c1 = 0.0f, c2 = 0.0f;
            for (int j = n_j - 1; j >= 0; --j) {
                float4 c = tn[j];
                float bj = fmaf(fmaf(c.y, x, c.x), c1, fmaf(c.z, c2, c.w));
                c2 = c1;
                c1 = bj;
            }
            float qq = q * q;
            float pw = qq * qq;
            for (int m = 0; m < n; ++m) pw *= q;
            out[n] = (b2 * pw) * c1;
        }
    }
}

__global__ void __launch_bounds__(GS_THREADS) gim_zi_kernel(GimArgs A, const float *atab, int n_in, int n_edge)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    const int NP1 = A.N + 1;
    const int nz = n_in + n_edge;
    float *stab = reinterpret_cast<float *>(dsm);   // [nz][N+1]
    float *salpha = stab + nz * NP1;                // [N+1][GS_THREADS]
    __shared__ GeomRec srec;
    __shared__ int sitem, sgeom, sfirst, scount, sbad;

    const int nss = A.n_ss;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int total = A.pref[A.n_geom];
    const float inv_nss = 1.0f / (float)nss;
    int nbad = 0;
    int staged = -1;
    if (tid == 0) sbad = 0;

#pragma unroll 1
    for (;;) {
        if (warp == 0) {
            int it = 0;
            if (lane == 0) it = atomicAdd(A.ctr, 1);
            it = __shfl_sync(0xffffffffu, it, 0);
            if (it < total) {
                const int pos = item_geometry(A.pref, A.n_geom, it, lane);
                if (lane == 0) {
                    const int g = A.gord[pos];
                    sgeom = g;
                    sfirst = A.pref[pos];
                    scount = A.cnt[g];
                }
            }
            if (lane == 0) sitem = it;
        }
        __syncthreads();
        const int it = sitem;
        const int g = sgeom;
        if (it >= total) break;   // uniform over the CTA
        if (g != staged) {
            const float *src = atab + (size_t)g * nz * NP1;
            for (int i = tid; i < nz * NP1; i += GS_THREADS) stab[i] = src[i];
            if (tid < 6) reinterpret_cast<float4 *>(&srec)[tid] = reinterpret_cast<const float4 *>(&A.rec[g])[tid];
            staged = g;
        }
        for (int n = 0; n < NP1; ++n) salpha[n * GS_THREADS + tid] = 0.0f;
        __syncthreads();
        const int i = (it - sfirst) * GS_THREADS + tid;
        if (i < scount) {
            const int t = A.list[(size_t)g * A.n_t + i];
            float2 ts = A.tsplit[t];
            float dt = pt::reduce_time(ts.x, ts.y, srec);
            const float kk = srec.k;
            const ZiGrid G = zi_grid(kk, n_in, n_edge);
            float warm[3] = {__int_as_float(0x7fffffff), 0.0f, 0.0f};   // Kepler warm start (none yet)
#pragma unroll 1
            for (int s = 0; s < nss; ++s) {
                bool bad = false;
                float z = pt::orbit_z<true>(srec, dt + ss_offset(A.t_exp, s, inv_nss), A.max_iter, &bad, warm);
                if (bad) ++nbad;
                if (!(z < 1.0f + kk)) continue;   // out of transit: alpha = 0
                int i0;
                float w;
                if (z <= G.zb && G.zb > 0.0f) {
                    float f = z * G.inv_h1;
                    i0 = min((int)f, n_in - 2);
                    w = f - (float)i0;
                } else if (z <= G.zb) {            // k >= 1: the first region is z = 0
                    i0 = 0;
                    w = 0.0f;
                } else {
                    float f = (z - G.zb) * G.inv_h2;
                    int c = min((int)f, n_edge - 1);
                    i0 = n_in - 1 + c;
                    w = f - (float)c;
                }
                const float *a0 = stab + i0 * NP1;
                for (int n = 0; n < NP1; ++n)
                    salpha[n * GS_THREADS + tid] += fmaf(w, a0[NP1 + n] - a0[n], a0[n]);
            }
#pragma unroll 1
            for (int bb = 0; bb < A.n_bpg; ++bb) {
                size_t row = (size_t)g * A.n_bpg + bb;
                const float *u = A.ld + row * A.N;
                // C_0 = (1 - sum u)/D, C_n = u_n/D, D = 1 - sum n u_n/(n+2)   (Sec. 2.1.3)
                float su = 0.0f, sd = 0.0f;
                for (int n = 1; n <= A.N; ++n) {
                    float un = u[n - 1];
                    su += un;
                    sd += (float)n * un / (float)(n + 2);
                }
                float al = (1.0f - su) * salpha[tid];
                for (int n = 1; n <= A.N; ++n) al = fmaf(u[n - 1], salpha[n * GS_THREADS + tid], al);
                A.flux[row * A.n_t + t] = 1.0f - al / (1.0f - sd) * inv_nss;
            }
        }
    }
    if (nbad) atomicAdd(&sbad, nbad);
    __syncthreads();
    if (tid == 0 && sbad && A.n_bad) atomicAdd(A.n_bad, sbad);
}

size_t gim_zi_smem(int N, int nz) { return (size_t)(N + 1) * (nz + GS_THREADS) * sizeof(float); }

// ---------------------------------------------------------------------------
// Mandel-Agol over the window kernel's pair lists: persistent CTAs take work
// items of MA_PPI listed (time, geometry) pairs.  An item runs in batches of
// up to MA_SSB supersamples:
//  1. each thread (one pair) computes z at the batch's supersamples and keeps
//     the in-transit ones (z < 1 + k) in order; a scan over the CTA places
//     every pair's z in one dense list, the supersamples with the planet
//     wholly inside the stellar disk (z <= 1 - k) first and those on the limb
//     after them, and records where each of its entries went;
//  2. each thread evaluates lambda_e, lambda_d + 2/3 Theta and eta_d at
//     entries tid, tid + MA_PPI, ... of the list, whatever pairs they belong
//     to: no lane idles on an out-of-transit supersample, and a warp mostly
//     takes one branch of the case table (the limb cases add the lens
//     geometry).  The terms go to shared memory;
//  3. each thread adds its own pair's terms in supersample order (the others
//     are zero), so the sums do not depend on where the terms were computed.
// Then the passband fluxes (Eq. ma_model).
// ---------------------------------------------------------------------------
constexpr int MA_PPI = 128;   // pairs per work item (= threads per CTA)
constexpr int MA_SSB = 16;    // supersamples per batch

__global__ void __launch_bounds__(MA_PPI, 8) ma_pairs_kernel(GimArgs A)
{
    __shared__ GeomRec srec;
    __shared__ int sitem, sgeom, sfirst, scount, sbad;
    __shared__ int swarp[MA_PPI / 32];
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int nss = A.n_ss;
    const int ssb = min(nss, MA_SSB);
    extern __shared__ __align__(16) unsigned char msm[];
    float *sT = reinterpret_cast<float *>(msm);                     // [3][ssb MA_PPI] terms of the list
    float *sz = sT + 3 * ssb * MA_PPI;                              // [ssb MA_PPI] the dense list of z
    float *szp = sz + ssb * MA_PPI;                                 // [ssb][MA_PPI] each pair's z, in order
    unsigned short *spos = reinterpret_cast<unsigned short *>(szp + ssb * MA_PPI);   // [ssb][MA_PPI] list slots
    const int total = A.pref[A.n_geom];
    const float inv_nss = 1.0f / (float)nss;
    int nbad = 0;
    int staged = -1;
    if (tid == 0) sbad = 0;
#pragma unroll 1
    for (;;) {
        if (warp == 0) {
            int it = 0;
            if (lane == 0) it = atomicAdd(A.ctr, 1);
            it = __shfl_sync(0xffffffffu, it, 0);
            if (it < total) {
                const int pos = item_geometry(A.pref, A.n_geom, it, lane);
                if (lane == 0) {
                    const int g = A.gord[pos];
                    sgeom = g;
                    sfirst = A.pref[pos];
                    scount = A.cnt[g];
                }
            }
            if (lane == 0) sitem = it;
        }
        __syncthreads();
        const int it = sitem;
        const int g = sgeom;
        if (it >= total) break;   // uniform over the CTA
        if (g != staged) {
            if (tid < 6) reinterpret_cast<float4 *>(&srec)[tid] = reinterpret_cast<const float4 *>(&A.rec[g])[tid];
            staged = g;
        }
        __syncthreads();
        const int i = (it - sfirst) * MA_PPI + tid;
        const bool own = i < scount;
        const int t = own ? A.list[(size_t)g * A.n_t + i] : 0;
        float dt = 0.0f;
        if (own) {
            const float2 ts = A.tsplit[t];
            dt = pt::reduce_time(ts.x, ts.y, srec);
        }
        const float kk = srec.k;
        float le = 0.0f, ld = 0.0f, ed = 0.0f;
        float warm[3] = {__int_as_float(0x7fffffff), 0.0f, 0.0f};   // Kepler warm start (none yet)
#pragma unroll 1
        for (int sb0 = 0; sb0 < nss; sb0 += ssb) {
            // 1. in-transit supersamples of this pair, in order (the terms of
            //    the others are zero: ma_terms returns zeros there), and which
            //    of them have the planet wholly inside the disk
            int c = 0, n_in = 0;
            unsigned limb = 0u;
            if (own) {
                const int s1 = min(nss, sb0 + ssb);
#pragma unroll 1
                for (int s = sb0; s < s1; ++s) {
                    bool bad = false;
                    const float z = pt::orbit_z<true, true>(srec, dt + ss_offset(A.t_exp, s, inv_nss), A.max_iter, &bad, warm);
                    if (bad) ++nbad;
                    if (z < 1.0f + kk && kk > 0.0f) {
                        szp[c * MA_PPI + tid] = z;
                        if ((z - 1.0f) + kk > 0.0f) limb |= 1u << c;
                        else ++n_in;
                        ++c;
                    }
                }
            }
            // both classes' counts in one scan: inside in the low 16 bits,
            // limb in the high ones (at most MA_SSB MA_PPI = 2048 each)
            const int v = n_in | ((c - n_in) << 16);
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) swarp[warp] = incl;
            __syncthreads();
            int base = 0, all = 0;
#pragma unroll
            for (int w = 0; w < MA_PPI / 32; ++w) {
                base += (w < warp) ? swarp[w] : 0;
                all += swarp[w];
            }
            const int excl = base + incl - v;
            const int n_inside = all & 0xffff;
            int p_in = excl & 0xffff, p_limb = n_inside + (excl >> 16);
            for (int j = 0; j < c; ++j) {
                const int pos = ((limb >> j) & 1u) ? p_limb++ : p_in++;
                sz[pos] = szp[j * MA_PPI + tid];
                spos[j * MA_PPI + tid] = (unsigned short)pos;
            }
            const int n_e = n_inside + (all >> 16);
            __syncthreads();
            // 2. the terms of every entry of the list
            const int stride = ssb * MA_PPI;
#pragma unroll 1
            for (int e = tid; e < n_e; e += MA_PPI) {
                float a0, a1, a2;
                pt::ma_terms(kk, sz[e], &a0, &a1, &a2);
                sT[e] = a0;
                sT[stride + e] = a1;
                sT[2 * stride + e] = a2;
            }
            __syncthreads();
            // 3. this pair's terms, in supersample order
            for (int j = 0; j < c; ++j) {
                const int pos = spos[j * MA_PPI + tid];
                le += sT[pos];
                ld += sT[stride + pos];
                ed += sT[2 * stride + pos];
            }
            __syncthreads();
        }
        if (own) {
            le *= inv_nss;
            ld *= inv_nss;
            ed *= inv_nss;
#pragma unroll 1
            for (int bb = 0; bb < A.n_bpg; ++bb) {
                size_t row = (size_t)g * A.n_bpg + bb;
                float we, wd, wn;
                pt::ma_weights(A.ld[row * 2], A.ld[row * 2 + 1], &we, &wd, &wn);
                A.flux[row * A.n_t + t] = 1.0f - (we * le + wd * ld + wn * ed);
            }
        }
    }
    if (nbad) atomicAdd(&sbad, nbad);
    __syncthreads();
    if (tid == 0 && sbad && A.n_bad) atomicAdd(A.n_bad, sbad);
}

// the list's terms, the list, each pair's z and the list slots
size_t ma_pairs_smem(int n_ss)
{
    const size_t n = (size_t)(n_ss < MA_SSB ? n_ss : MA_SSB) * MA_PPI;
    return n * (5 * sizeof(float) + sizeof(unsigned short));
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

// ssr[row] = sum_t wt (y - flux)^2 over one flux row, in a fixed order;
// row r observes passband r % n_b (rows are geometry-major, band-minor).
// ssr_part_kernel: one CTA per (row, chunk of SSR_CHUNK times); every thread
// loads its SSR_PER values before adding them, so a CTA keeps its whole chunk
// in flight (a loop that waits on each load in turn is latency-bound), then a
// fixed-order block sum.  ssr_reduce_kernel adds a row's chunk sums.
constexpr int SSR_PER = 16;
constexpr int SSR_CHUNK = 256 * SSR_PER;

int ssr_chunks(int n_t) { return (n_t + SSR_CHUNK - 1) / SSR_CHUNK; }

__global__ void __launch_bounds__(256) ssr_part_kernel(const float *flux, const float *y, const float *wt, int n_t,
                                                      int n_b, float *part)
{
    __shared__ float sred[8];
    const size_t row = blockIdx.x;
    const int band = (int)(row % n_b);
    const float *f = flux + row * n_t;
    const float *yb = y + (size_t)band * n_t;
    const float *wb = wt ? wt + (size_t)band * n_t : nullptr;
    const int t0 = blockIdx.y * SSR_CHUNK + threadIdx.x;
    float fv[SSR_PER], yv[SSR_PER], wv[SSR_PER];
#pragma unroll
    for (int j = 0; j < SSR_PER; ++j) {
        const int t = t0 + j * 256;
        const bool ok = t < n_t;
        fv[j] = ok ? f[t] : 0.0f;
        yv[j] = ok ? yb[t] : 0.0f;
        wv[j] = ok ? (wb ? wb[t] : 1.0f) : 0.0f;
    }
    float acc = 0.0f;
#pragma unroll
    for (int j = 0; j < SSR_PER; ++j) {
        const float r = yv[j] - fv[j];
        acc = fmaf(wv[j], r * r, acc);
    }
    const float tot = block_sum(acc, sred);
    if (threadIdx.x == 0) part[row * gridDim.y + blockIdx.y] = tot;
}

int launch_ssr_rows(const float *flux, const float *y, const float *wt, int n_t, int n_b, size_t rows, float *part,
                    float *ssr, cudaStream_t s)
{
    const int nc = ssr_chunks(n_t);
    ssr_part_kernel<<<dim3((unsigned)rows, (unsigned)nc), 256, 0, s>>>(flux, y, wt, n_t, n_b, part);
    int st = check_launch("ssr_part_kernel");
    if (st) return st;
    ssr_reduce_kernel<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(part, (int)rows, nc, ssr);
    return check_launch("ssr_reduce_kernel");
}

// Interpolation-table nodes: the exact FP32 terms at (k_i, z_j), positions
// formed in FP64 and rounded once.
__global__ void ma_table_kernel(double k_lo, double k_hi, int n_k, int n_z, float4 *tab)
{
    size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (size_t)n_k * n_z) return;
    int i = (int)(id / n_z), j = (int)(id % n_z);
    float k = (float)(k_lo + i * (k_hi - k_lo) / (n_k - 1));
    float z = (float)(j * (1.0 + k_hi) / (n_z - 1));
    float le, ld, ed;
    pt::ma_terms(k, z, &le, &ld, &ed);
    tab[id] = make_float4(le, ld, ed, 0.0f);
}

__global__ void ma_terms_interp_kernel(const float4 *tab, int n_k, int n_z, float k_lo, float k_hi, float inv_dk,
                                       float inv_dz, const float *k, const float *z, size_t n, float *le, float *ld,
                                       float *ed)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float a, b, c;
    pt::ma_interp(tab, n_k, n_z, k_lo, k_hi, inv_dk, inv_dz, k[i], z[i], &a, &b, &c);
    if (le) le[i] = a;
    if (ld) ld[i] = b;
    if (ed) ed[i] = c;
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

// Exposure time: finite and non-negative (the supersamples of Sec. 3.2 span it).
bool exposure_ok(double t_exp) { return t_exp >= 0.0 && t_exp < 1.0e30; }

int check_orbit(const pt_orbit *orb, bool need_ecc)
{
    if (!orb || orb->n_v < 0) return PT_ERR_ARG;
    if (orb->n_v == 0) return PT_OK;
    if (!orb->t0 || !orb->P || !orb->a || !orb->inc) return PT_ERR_ARG;
    if ((orb->e == nullptr) != (orb->w == nullptr)) return PT_ERR_ARG;
    if (need_ecc && !orb->e) return PT_ERR_ARG;
    return PT_OK;
}

// Mandel-Agol (NP1 == 0): records, time split, per-tile residual partials.
// Gimenez: records, time split, per-geometry tables, list counters (+ the
// work-item counter), work-item prefix, pair lists and a flux scratch used
// when only residuals are asked for.
struct WorkLayout {
    size_t rec, tsplit, T, part, cnt, pref, list, fscr, atab, dtab, total;
};

// n_zi > 0 adds the z tables of the interpolated Gimenez model.
WorkLayout work_layout(int n_t, int n_v, int n_b, int k_per_band, int NP1, int n_j, int n_zi = 0)
{
    int n_geom = k_per_band ? n_v * n_b : n_v;
    int n_tiles = (n_t + TT - 1) / TT;
    WorkLayout L;
    size_t off = 0;
    L.rec = off;
    off += align256((size_t)n_geom * sizeof(GeomRec));
    L.tsplit = off;
    off += align256((size_t)n_t * sizeof(float2));
    L.T = L.part = L.cnt = L.pref = L.list = L.fscr = L.atab = L.dtab = off;
    if (NP1 == 0) {
        L.part = off;
        off += align256((size_t)n_v * n_b * n_tiles * sizeof(float));
    } else {
        L.T = off;
        off += align256((size_t)n_geom * NP1 * n_j * sizeof(float4));
        L.cnt = off;
        off += align256((size_t)(n_geom + 1) * sizeof(int));
        L.pref = off;   // the item prefix [n_geom + 1], then the geometry order [n_geom]
        off += align256((size_t)(2 * n_geom + 1) * sizeof(int));
        L.list = off;
        off += align256((size_t)n_geom * n_t * sizeof(int));
        L.fscr = off;
        off += align256((size_t)n_v * n_b * n_t * sizeof(float));
        L.part = off;   // residual chunk sums
        off += align256((size_t)n_v * n_b * ssr_chunks(n_t) * sizeof(float));
        L.atab = off;
        off += align256((size_t)n_geom * n_zi * NP1 * sizeof(float));
        L.dtab = off;   // Chebyshev coefficient rows, padded to 16 bytes
        off += align256((size_t)n_geom * n_j * ((NP1 + 3) & ~3) * sizeof(float));
    }
    L.total = off;
    return L;
}

// pt_ma_quad runs over the window kernel's pair lists (the list layout: no
// Gimenez tables), except for a few geometries: there the tile kernel's two
// launches (set-up, evaluation) beat the list path's four (one light curve
// of 1,000 points: 12.3 against 16.4 us per CUDA-graph replay; the list path
// wins from about 16 geometries).  The tile kernel also serves the
// interpolated and the allocation-free variants.
constexpr bool MA_LIST = true;
constexpr int MA_TILE_MAX_GEOM = 4;

bool ma_small(const pt_orbit *orb, int n_b, int k_per_band)
{
    if (!orb || orb->n_v < 0 || n_b < 1) return false;
    const long long n_geom = k_per_band ? (long long)orb->n_v * n_b : orb->n_v;
    return n_geom <= MA_TILE_MAX_GEOM;
}

size_t ma_list_work_bytes(int n_t, int n_v, int n_b, int k_per_band)
{
    return work_layout(n_t, n_v, n_b, k_per_band, 1, 0).total;
}

}  // namespace

struct pt_ma_table_s {
    float k_lo, k_hi, inv_dk, inv_dz;
    int n_k, n_z;
    float4 *d_tab;   // [n_k][n_z]: (lambda_e, lambda_d + 2/3 Theta, eta_d, 0)
};

// The table's device view, for the batched path (pt_batch.cu).
namespace pt_internal {
bool ma_table_view(pt_ma_table t, const float4 **tab, int *n_k, int *n_z, float *k_lo, float *k_hi, float *inv_dk,
                   float *inv_dz)
{
    if (!t || !t->d_tab) return false;
    *tab = t->d_tab;
    *n_k = t->n_k;
    *n_z = t->n_z;
    *k_lo = t->k_lo;
    *k_hi = t->k_hi;
    *inv_dk = t->inv_dk;
    *inv_dz = t->inv_dz;
    return true;
}
}  // namespace pt_internal

struct pt_gim_plan_s {
    int N, n_j;
    float4 *d_coef;   // [N+1][n_j]: recursion of G_j(nu+2, 1; x), FP32
    double *d_A;      // [N+1][n_j]: A_{n,j}, FP64
    double *d_recb;   // [N+1][n_j][3]: recursion of G_j(nu+2, nu+1; x), FP64
    cudaEvent_t ev0, ev1;   // recorded around the series evaluation kernel when set (profiling)
    // The table recursion and the Chebyshev coefficients depend on k alone:
    // they run on this plan-owned stream (highest priority) beside the
    // set-up, window and scan kernels of the call's stream, forked and joined
    // by the two events; the mutex keeps a fork's record and wait together
    // when host threads share the plan.
    cudaStream_t side;
    cudaEvent_t ev_fork, ev_join;
    std::mutex fork_mu;
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
int launch_zi(const GimArgs &A, const float *atab, int n_in, int n_edge, size_t smem, size_t max_items,
              cudaStream_t s)
{
    static thread_local size_t configured = 0;
    if (smem > 48 * 1024 && smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(gim_zi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return set_cuda_error(e, "gim_zi_kernel smem attribute");
        configured = smem;
    }
    int dev = 0, n_sm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gim_zi_kernel, GS_THREADS, smem);
    if (e != cudaSuccess) return set_cuda_error(e, "gim_zi_kernel occupancy");
    if (per_sm < 1) return pt_internal::set_error(PT_ERR_ARG, "gim_zi_kernel", "does not fit on an SM");
    size_t grid = (size_t)n_sm * per_sm;
    if (grid > max_items) grid = max_items;
    if (grid < 1) grid = 1;
    gim_zi_kernel<<<(unsigned)grid, GS_THREADS, smem, s>>>(A, atab, n_in, n_edge);
    return check_launch("gim_zi_kernel");
}

// Chebyshev path, coefficient kernel for N + 1 orders.
template <int NP1>
int launch_cheb_coef_t(const GimArgs &A, const float4 *T, float *dtab, cudaStream_t s)
{
    // coefficients: one warp per (geometry, order), rows padded to DS
    // floats (the warps past order N write the padding zeros)
    constexpr int DS = (NP1 + 3) & ~3;
    const size_t csm = (size_t)CW_WARPS * A.n_j * sizeof(float4);
    const dim3 cgrid(A.n_geom, (DS + CW_WARPS - 1) / CW_WARPS);
    const int S = gim_cheb_coef_s(A.n_j);
#define PT_COEF_LAUNCH(SV)                                                                                          \
    gim_cheb_coef_kernel<SV><<<cgrid, 32 * CW_WARPS, csm, s>>>(T, A.N + 1, A.n_j, DS, dtab)
    if (S <= 2) PT_COEF_LAUNCH(2);
    else if (S <= 4) PT_COEF_LAUNCH(4);
    else if (S <= 6) PT_COEF_LAUNCH(6);
    else if (S <= 8) PT_COEF_LAUNCH(8);
    else if (S <= 12) PT_COEF_LAUNCH(12);
    else PT_COEF_LAUNCH(16);
#undef PT_COEF_LAUNCH
    return check_launch("gim_cheb_coef_kernel");
}

// Chebyshev path, evaluation kernel (persistent) for N + 1 orders.
template <int NP1>
int launch_cheb_eval_t(const GimArgs &A, float *dtab, size_t max_items, cudaEvent_t ev0, cudaEvent_t ev1,
                       cudaStream_t s)
{
    int st = PT_OK;
    // evaluation: persistent
    const size_t smem = gim_cheb_smem(A.n_j, A.N, A.n_ss);
    static thread_local size_t configured = 0;
    if (smem > 48 * 1024 && smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(gim_cheb_kernel<NP1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return set_cuda_error(e, "gim_cheb_kernel smem attribute");
        configured = smem;
    }
    int dev = 0, n_sm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gim_cheb_kernel<NP1>, GS_THREADS, smem);
    if (e != cudaSuccess) return set_cuda_error(e, "gim_cheb_kernel occupancy");
    if (per_sm < 1) return pt_internal::set_error(PT_ERR_ARG, "gim_cheb_kernel", "does not fit on an SM");
    size_t grid = (size_t)n_sm * per_sm;
    if (grid > max_items) grid = max_items;
    if (grid < 1) grid = 1;
    if (ev0 && (e = cudaEventRecord(ev0, s)) != cudaSuccess) return set_cuda_error(e, "pt_gimenez timing event");
    gim_cheb_kernel<NP1><<<(unsigned)grid, GS_THREADS, smem, s>>>(A, dtab);
    st = check_launch("gim_cheb_kernel");
    if (st) return st;
    if (ev1 && (e = cudaEventRecord(ev1, s)) != cudaSuccess) return set_cuda_error(e, "pt_gimenez timing event");
    return PT_OK;
}

// Chebyshev path dispatch over N + 1 = 2 .. 17 orders.
#define PT_NP1_DISPATCH(CALL)                                                                                       \
    switch (A.N + 1) {                                                                                              \
    case 2: return CALL(2);                                                                                         \
    case 3: return CALL(3);                                                                                         \
    case 4: return CALL(4);                                                                                         \
    case 5: return CALL(5);                                                                                         \
    case 6: return CALL(6);                                                                                         \
    case 7: return CALL(7);                                                                                         \
    case 8: return CALL(8);                                                                                         \
    case 9: return CALL(9);                                                                                         \
    case 10: return CALL(10);                                                                                       \
    case 11: return CALL(11);                                                                                       \
    case 12: return CALL(12);                                                                                       \
    case 13: return CALL(13);                                                                                       \
    case 14: return CALL(14);                                                                                       \
    case 15: return CALL(15);                                                                                       \
    case 16: return CALL(16);                                                                                       \
    default: return CALL(17);                                                                                       \
    }

int launch_cheb_coef(const GimArgs &A, const float4 *T, float *dtab, cudaStream_t s)
{
#define PT_CALL(V) launch_cheb_coef_t<V>(A, T, dtab, s)
    PT_NP1_DISPATCH(PT_CALL)
#undef PT_CALL
}

int launch_cheb_eval(const GimArgs &A, float *dtab, size_t max_items, cudaEvent_t ev0, cudaEvent_t ev1,
                     cudaStream_t s)
{
#define PT_CALL(V) launch_cheb_eval_t<V>(A, dtab, max_items, ev0, ev1, s)
    PT_NP1_DISPATCH(PT_CALL)
#undef PT_CALL
}
#undef PT_NP1_DISPATCH

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
// Parameter domain (include/pt.h, pt_domain_check): counts the geometries
// (vector, or vector and passband when k is per passband) whose parameters
// lie outside it.  Reads its inputs only.
__global__ void domain_kernel(const double *t0, const double *P, const float *a, const float *inc, const float *e,
                              const float *w, const float *k, int n_v, int n_kv, int *n_out)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (g < n_v * n_kv) {
        int v = g / n_kv;
        const float kk = k[g];
        bad = !(kk > 0.0f && kk <= 1.0e3f);
        if (g % n_kv == 0) {
            const double tv = t0[v], pv = P[v];
            const float av = a[v], iv = inc[v];
            bad |= !(fabs(tv) < 1.0e15) || !(pv > 0.0 && pv < 1.0e15) || !(av > 1.0f && av < 1.0e7f) ||
                   !(iv >= 0.0f && iv <= 3.14159274f);
            if (e) {
                const float ev = e[v], wv = w[v];
                bad |= !(ev >= 0.0f && ev <= 0.95f) || !(fabsf(wv) < 1.0e6f);
            }
        }
    }
    const unsigned m = __ballot_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(n_out, __popc(m));
}

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
    if (!exposure_ok(t_exp)) return pt_internal::set_error(PT_ERR_DOMAIN, "pt_z_circ", "exposure time must be finite and >= 0");
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
    if (!exposure_ok(t_exp)) return pt_internal::set_error(PT_ERR_DOMAIN, "pt_z_ecc", "exposure time must be finite and >= 0");
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

int pt_domain_check(const pt_orbit *orb, const float *k, int n_k_per_v, int *n_out, pt_stream_t stream)
{
    int st = check_orbit(orb, false);
    if (st) return st;
    if (n_k_per_v < 1 || !n_out) return PT_ERR_ARG;
    if (orb->n_v == 0) return PT_OK;
    if (!k || (long long)orb->n_v * n_k_per_v > 0x7fffffffLL) return PT_ERR_ARG;
    const int n = orb->n_v * n_k_per_v;
    domain_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(orb->t0, orb->P, orb->a, orb->inc, orb->e,
                                                                    orb->w, k, orb->n_v, n_k_per_v, n_out);
    return check_launch("pt_domain_check");
}

int pt_status_read(const int *n_bad, const int *n_domain, pt_stream_t stream)
{
    int h[2] = {0, 0};
    cudaStream_t s = (cudaStream_t)stream;
    const int *src[2] = {n_domain, n_bad};
    for (int i = 0; i < 2; ++i) {
        if (!src[i]) continue;
        cudaError_t e = cudaMemcpyAsync(&h[i], src[i], sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return set_cuda_error(e, "pt_status_read");
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_cuda_error(e, "pt_status_read");
    if (h[0] > 0) {
        snprintf(g_last_error, sizeof(g_last_error), "pt_status_read: %d geometries outside the parameter domain",
                 h[0]);
        return PT_ERR_DOMAIN;
    }
    if (h[1] > 0) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "pt_status_read: %d Newton solves stopped at the step cap before converging", h[1]);
        return PT_ERR_NOT_CONVERGED;
    }
    return PT_OK;
}

static int lc_common_check(const double *t, int n_t, const pt_orbit *orb, const float *k, int k_per_band,
                           const float *ld, int n_b, int n_ss, double t_exp, int max_iter, const float *y,
                           float *flux, float *ssr, void *work)
{
    int st = check_orbit(orb, false);
    if (st) return st;
    if (n_t < 0 || n_b < 1 || n_ss < 1 || n_ss > MAX_SS || max_iter < 1 || max_iter > MAX_NEWTON)
        return PT_ERR_ARG;
    if (k_per_band != 0 && k_per_band != 1) return PT_ERR_ARG;
    if (!exposure_ok(t_exp))
        return pt_internal::set_error(PT_ERR_DOMAIN, "light curve", "exposure time must be finite and >= 0");
    if (n_t == 0 || orb->n_v == 0) return PT_OK;   // nothing to evaluate
    if (!flux && !ssr) return PT_ERR_ARG;
    if (!t || !k || !ld) return PT_ERR_ARG;
    if (ssr && !y) return PT_ERR_ARG;
    if (!work || ((uintptr_t)work & 15u)) return PT_ERR_WORKSPACE;
    return PT_OK;
}

size_t pt_ma_quad_work_bytes(int n_t, int n_v, int n_b, int k_per_band)
{
    if (n_t < 0 || n_v < 0 || n_b < 1) return 0;
    size_t tile = work_layout(n_t, n_v, n_b, k_per_band, 0, 0).total;
    return MA_LIST ? ma_list_work_bytes(n_t, n_v, n_b, k_per_band) : tile;
}

static int launch_setup(const double *t, int n_t, const pt_orbit *orb, const float *k, int k_per_band, int n_b,
                        double t_exp, GeomRec *rec, float2 *tsplit, int *cnt, cudaStream_t s)
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
    sa.cnt = cnt;
    sa.half_exp = (float)(0.5 * t_exp);
    const int bs = 64;
    sa.n_gblocks = (sa.n_geom + bs - 1) / bs;
    int n_tblocks = (n_t + bs - 1) / bs;
    setup_kernel<<<sa.n_gblocks + n_tblocks, bs, 0, s>>>(sa);
    return check_launch("setup_kernel");
}

}  // extern "C"

// pt_ma_quad over the pair lists (window kernel, scan, ma_pairs_kernel).
static int ma_quad_list(const double *t, int n_t, const pt_orbit *orb, const float *k, int k_per_band,
                        const float *ld, int n_b, int n_ss, double t_exp, int max_iter, const float *y,
                        const float *wt, float *flux, float *ssr, void *work, size_t work_bytes, int *n_bad,
                        pt_stream_t stream)
{
    int st = lc_common_check(t, n_t, orb, k, k_per_band, ld, n_b, n_ss, t_exp, max_iter, y, flux, ssr, work);
    if (st) return st;
    if (n_t == 0 || orb->n_v == 0) return PT_OK;
    WorkLayout L = work_layout(n_t, orb->n_v, n_b, k_per_band, 1, 0);
    if (work_bytes < L.total) return PT_ERR_WORKSPACE;
    const int n_geom = k_per_band ? orb->n_v * n_b : orb->n_v;
    const int n_tiles = (n_t + TT - 1) / TT;
    const int gy = (n_geom + GW_VT - 1) / GW_VT;
    if (gy > 65535) return PT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    char *wb = (char *)work;
    GeomRec *rec = (GeomRec *)(wb + L.rec);
    float2 *tsplit = (float2 *)(wb + L.tsplit);
    int *cnt = (int *)(wb + L.cnt);
    st = launch_setup(t, n_t, orb, k, k_per_band, n_b, t_exp, rec, tsplit, cnt, s);
    if (st) return st;
    GimArgs A;
    memset(&A, 0, sizeof(A));
    A.tsplit = tsplit;
    A.n_t = n_t;
    A.rec = rec;
    A.n_geom = n_geom;
    A.ld = ld;
    A.N = 2;
    A.n_bpg = k_per_band ? 1 : n_b;
    A.n_ss = n_ss;
    A.t_exp = (float)t_exp;
    A.max_iter = max_iter;
    A.flux = flux ? flux : (float *)(wb + L.fscr);
    A.cnt = cnt;
    A.pref = (int *)(wb + L.pref);
    A.gord = A.pref + n_geom + 1;
    A.ctr = cnt + n_geom;
    A.list = (int *)(wb + L.list);
    A.ppi = MA_PPI;
    A.n_bad = n_bad;
    TableJob J;
    memset(&J, 0, sizeof(J));
    const size_t n_cta = (size_t)n_tiles * gy;
    if (n_cta > 0x7fffffffULL) return PT_ERR_ARG;
    gim_window_kernel<<<(unsigned)n_cta, TT, 0, s>>>(A, J, n_tiles);
    st = check_launch("gim_window_kernel");
    if (st) return st;
    gim_scan_kernel<<<1, 1024, 0, s>>>(cnt, A.rec, A.t_exp, n_geom, MA_PPI, false, A.pref, A.gord, A.ctr);
    st = check_launch("gim_scan_kernel");
    if (st) return st;
    const size_t msm = ma_pairs_smem(n_ss);   // at most 44 KB: no opt-in needed
    int dev = 0, n_sm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ma_pairs_kernel, MA_PPI, msm);
    if (e != cudaSuccess) return set_cuda_error(e, "ma_pairs_kernel occupancy");
    size_t grid = (size_t)n_sm * (per_sm > 0 ? per_sm : 1);
    const size_t max_items = (size_t)n_geom * ((n_t + MA_PPI - 1) / MA_PPI);
    if (grid > max_items) grid = max_items;
    if (grid < 1) grid = 1;
    ma_pairs_kernel<<<(unsigned)grid, MA_PPI, msm, s>>>(A);
    st = check_launch("ma_pairs_kernel");
    if (st) return st;
    if (ssr) st = launch_ssr_rows(A.flux, y, wt, n_t, n_b, (size_t)orb->n_v * n_b, (float *)(wb + L.part), ssr, s);
    return st;
}

// pt_ma_quad and pt_ma_quad_interp: exact terms when tab is null, else the
// interpolated ones.
static int ma_quad_impl(const pt_ma_table_s *tab, const double *t, int n_t, const pt_orbit *orb, const float *k,
                        int k_per_band, const float *ld, int n_b, int n_ss, double t_exp, int max_iter,
                        const float *y, const float *wt, float *flux, float *ssr, void *work, size_t work_bytes,
                        int *n_bad, pt_stream_t stream)
{
    int st = lc_common_check(t, n_t, orb, k, k_per_band, ld, n_b, n_ss, t_exp, max_iter, y, flux, ssr, work);
    if (st) return st;
    if (n_t == 0 || orb->n_v == 0) return PT_OK;
    WorkLayout L = work_layout(n_t, orb->n_v, n_b, k_per_band, 0, 0);
    if (work_bytes < L.total) return PT_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    char *wb = (char *)work;
    GeomRec *rec = (GeomRec *)(wb + L.rec);
    float2 *tsplit = (float2 *)(wb + L.tsplit);
    float *part = (float *)(wb + L.part);
    st = launch_setup(t, n_t, orb, k, k_per_band, n_b, t_exp, rec, tsplit, nullptr, s);
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
    if (tab) {
        A.mtab = tab->d_tab;
        A.mn_k = tab->n_k;
        A.mn_z = tab->n_z;
        A.mk_lo = tab->k_lo;
        A.mk_hi = tab->k_hi;
        A.minv_dk = tab->inv_dk;
        A.minv_dz = tab->inv_dz;
        ma_lc_kernel<true><<<grid, TT, 0, s>>>(A);
    } else {
        ma_lc_kernel<false><<<grid, TT, 0, s>>>(A);
    }
    st = check_launch("ma_lc_kernel");
    if (st) return st;
    if (ssr) {
        int rows = orb->n_v * n_b;
        ssr_reduce_kernel<<<(rows * 32 + 255) / 256, 256, 0, s>>>(part, rows, A.n_tiles, ssr);
        st = check_launch("ssr_reduce_kernel");
    }
    return st;
}

extern "C" {

int pt_ma_quad(const double *t, int n_t, const pt_orbit *orb, const float *k, int k_per_band, const float *ld,
               int n_b, int n_ss, double t_exp, int max_iter, const float *y, const float *wt, float *flux,
               float *ssr, void *work, size_t work_bytes, int *n_bad, pt_stream_t stream)
{
    if (MA_LIST && !ma_small(orb, n_b, k_per_band))
        return ma_quad_list(t, n_t, orb, k, k_per_band, ld, n_b, n_ss, t_exp, max_iter, y, wt, flux, ssr, work,
                            work_bytes, n_bad, stream);
    return ma_quad_impl(nullptr, t, n_t, orb, k, k_per_band, ld, n_b, n_ss, t_exp, max_iter, y, wt, flux, ssr,
                        work, work_bytes, n_bad, stream);
}

int pt_ma_quad_interp(pt_ma_table table, const double *t, int n_t, const pt_orbit *orb, const float *k,
                      int k_per_band, const float *ld, int n_b, int n_ss, double t_exp, int max_iter, const float *y,
                      const float *wt, float *flux, float *ssr, void *work, size_t work_bytes, int *n_bad,
                      pt_stream_t stream)
{
    if (!table) return PT_ERR_ARG;
    return ma_quad_impl(table, t, n_t, orb, k, k_per_band, ld, n_b, n_ss, t_exp, max_iter, y, wt, flux, ssr, work,
                        work_bytes, n_bad, stream);
}

int pt_ma_table_create(float k_lo, float k_hi, int n_k, int n_z, pt_ma_table *out)
{
    if (!out) return PT_ERR_ARG;
    *out = nullptr;
    if (!(k_lo > 0.0f) || !(k_hi > k_lo) || n_k < 2 || n_k > 4096 || n_z < 2 || n_z > 65536) return PT_ERR_ARG;
    pt_ma_table p = new pt_ma_table_s;
    p->k_lo = k_lo;
    p->k_hi = k_hi;
    p->n_k = n_k;
    p->n_z = n_z;
    p->inv_dk = (float)((n_k - 1) / ((double)k_hi - (double)k_lo));
    p->inv_dz = (float)((n_z - 1) / (1.0 + (double)k_hi));
    p->d_tab = nullptr;
    size_t cnt = (size_t)n_k * n_z;
    cudaError_t e = cudaMalloc(&p->d_tab, cnt * sizeof(float4));
    if (e == cudaSuccess) {
        ma_table_kernel<<<(unsigned)((cnt + 255) / 256), 256>>>(k_lo, k_hi, n_k, n_z, p->d_tab);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(p->d_tab);
        delete p;
        return set_cuda_error(e, "pt_ma_table_create");
    }
    *out = p;
    return PT_OK;
}

int pt_ma_table_destroy(pt_ma_table p)
{
    if (!p) return PT_OK;
    cudaFree(p->d_tab);
    delete p;
    return PT_OK;
}

int pt_ma_terms_interp(pt_ma_table p, const float *k, const float *z, size_t n, float *le, float *ld, float *ed,
                       pt_stream_t stream)
{
    if (!p) return PT_ERR_ARG;
    if (n == 0) return PT_OK;
    if (!k || !z) return PT_ERR_ARG;
    size_t blocks = (n + 255) / 256;
    if (blocks > 0x7fffffffULL) return PT_ERR_ARG;
    ma_terms_interp_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
        p->d_tab, p->n_k, p->n_z, p->k_lo, p->k_hi, p->inv_dk, p->inv_dz, k, z, n, le, ld, ed);
    return check_launch("pt_ma_terms_interp");
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
    p->ev0 = p->ev1 = nullptr;
    p->side = nullptr;
    p->ev_fork = p->ev_join = nullptr;
    int prio_lo = 0, prio_hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&p->side, cudaStreamNonBlocking, prio_hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_coef, cnt * sizeof(float4));
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
        if (p->ev_fork) cudaEventDestroy(p->ev_fork);
        if (p->ev_join) cudaEventDestroy(p->ev_join);
        if (p->side) cudaStreamDestroy(p->side);
        delete p;
        return set_cuda_error(e, "pt_gim_plan_create");
    }
    *out = p;
    return PT_OK;
}

int pt_gim_plan_time_evaluation(pt_gim_plan p, void *ev_start, void *ev_end)
{
    if (!p || (ev_start == nullptr) != (ev_end == nullptr)) return PT_ERR_ARG;
    p->ev0 = (cudaEvent_t)ev_start;
    p->ev1 = (cudaEvent_t)ev_end;
    return PT_OK;
}

int pt_gim_plan_destroy(pt_gim_plan p)
{
    if (!p) return PT_OK;
    cudaFree(p->d_coef);
    cudaFree(p->d_A);
    cudaFree(p->d_recb);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    if (p->side) cudaStreamDestroy(p->side);
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

}  // extern "C"

// pt_gimenez (n_in == 0: the series for every pair) and pt_gimenez_zi (the
// series on z nodes, read back by interpolation).
static int gimenez_impl(pt_gim_plan plan, int n_in, int n_edge, const double *t, int n_t, const pt_orbit *orb,
                        const float *k, int k_per_band, const float *ld, int n_b, int n_ss, double t_exp,
                        int max_iter, const float *y, const float *wt, float *flux, float *ssr, void *work,
                        size_t work_bytes, int *n_bad, pt_stream_t stream)
{
    if (!plan) return PT_ERR_ARG;
    const bool zi = n_in > 0;
    if (zi && (n_in < 2 || n_edge < 1 || (size_t)(n_in + n_edge) * (plan->N + 1) > (size_t)ZI_MAX_VALUES))
        return PT_ERR_ARG;
    int st = lc_common_check(t, n_t, orb, k, k_per_band, ld, n_b, n_ss, t_exp, max_iter, y, flux, ssr, work);
    if (st) return st;
    if (n_t == 0 || orb->n_v == 0) return PT_OK;
    const int NP1 = plan->N + 1;
    WorkLayout L = work_layout(n_t, orb->n_v, n_b, k_per_band, NP1, plan->n_j, zi ? n_in + n_edge : 0);
    if (work_bytes < L.total) return PT_ERR_WORKSPACE;
    const size_t smem = zi ? gim_zi_smem(plan->N, n_in + n_edge) : gim_cheb_smem(plan->n_j, plan->N, n_ss);
    if (smem > 200 * 1024) return PT_ERR_ARG;
    const int n_geom = k_per_band ? orb->n_v * n_b : orb->n_v;
    const int n_tiles = (n_t + TT - 1) / TT;
    const int gy = (n_geom + GW_VT - 1) / GW_VT;
    if (gy > 65535) return PT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    char *wb = (char *)work;
    GeomRec *rec = (GeomRec *)(wb + L.rec);
    float2 *tsplit = (float2 *)(wb + L.tsplit);
    float4 *T = (float4 *)(wb + L.T);
    int *cnt = (int *)(wb + L.cnt);
    float *atab = (float *)(wb + L.atab);
    float *dtab = (float *)(wb + L.dtab);
    GimArgs A;
    memset(&A, 0, sizeof(A));
    A.tsplit = tsplit;
    A.n_t = n_t;
    A.rec = rec;
    A.n_geom = n_geom;
    A.gtab = T;
    A.N = plan->N;
    A.n_j = plan->n_j;
    A.ld = ld;
    A.n_bpg = k_per_band ? 1 : n_b;
    A.n_ss = n_ss;
    A.t_exp = (float)t_exp;
    A.max_iter = max_iter;
    A.flux = flux ? flux : (float *)(wb + L.fscr);
    A.cnt = cnt;
    A.pref = (int *)(wb + L.pref);
    A.gord = A.pref + n_geom + 1;
    A.ctr = cnt + n_geom;
    A.list = (int *)(wb + L.list);
    A.ppi = GS_THREADS;   // work items of GS_THREADS listed pairs
    A.n_bad = n_bad;
    TableJob J;
    J.k = k;
    J.n_geom = n_geom;
    J.NP1 = NP1;
    J.n_j = plan->n_j;
    J.A = plan->d_A;
    J.recb = plan->d_recb;
    J.coef = plan->d_coef;
    J.tab = T;
    J.n_blocks = NP1 * ((n_geom + TABLE_GPC - 1) / TABLE_GPC);
    const size_t tsm = gim_table_smem(plan->n_j);   // at most 24 KB (n_j <= 512): no opt-in needed
    if (!zi) {
        // the table recursion and the Chebyshev coefficients depend on k
        // alone: forked onto the plan's side stream (after all earlier work
        // of the call's stream), joined before the evaluation kernel
        cudaError_t e;
        {
            std::lock_guard<std::mutex> lk(plan->fork_mu);
            e = cudaEventRecord(plan->ev_fork, s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->side, plan->ev_fork, 0);
        }
        if (e != cudaSuccess) return set_cuda_error(e, "pt_gimenez fork");
        const size_t tsm2 = gim_table2_smem(plan->n_j);
        static thread_local size_t tsm2_configured = 0;
        if (tsm2 > 48 * 1024 && tsm2 > tsm2_configured) {
            e = cudaFuncSetAttribute(gim_table_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm2);
            if (e != cudaSuccess) return set_cuda_error(e, "gim_table_kernel smem attribute");
            tsm2_configured = tsm2;
        }
        const int n_tb = NP1 * ((n_geom + TABLE_GPC2 - 1) / TABLE_GPC2);
        gim_table_kernel<<<(unsigned)n_tb, TT, tsm2, plan->side>>>(J);
        st = check_launch("gim_table_kernel");
        if (st) return st;
        st = launch_cheb_coef(A, T, dtab, plan->side);
        if (st) return st;
        e = cudaEventRecord(plan->ev_join, plan->side);
        if (e != cudaSuccess) return set_cuda_error(e, "pt_gimenez join");
        J.n_blocks = 0;   // the window launch without table CTAs
    }
    st = launch_setup(t, n_t, orb, k, k_per_band, n_b, t_exp, rec, tsplit, cnt, s);
    if (st) return st;
    const size_t n_cta = (size_t)J.n_blocks + (size_t)n_tiles * gy;
    if (n_cta > 0x7fffffffULL) return PT_ERR_ARG;
    gim_window_kernel<<<(unsigned)n_cta, TT, J.n_blocks ? tsm : 0, s>>>(A, J, n_tiles);
    st = check_launch("gim_window_kernel");
    if (st) return st;
    if (zi) {
        gim_zi_table_kernel<<<n_geom, 128, 0, s>>>(rec, T, NP1, plan->n_j, n_in, n_edge, atab);
        st = check_launch("gim_zi_table_kernel");
        if (st) return st;
    }
    gim_scan_kernel<<<1, 1024, 0, s>>>(cnt, A.rec, A.t_exp, n_geom, A.ppi, true, A.pref, A.gord, A.ctr);
    st = check_launch("gim_scan_kernel");
    if (st) return st;
    const size_t max_items = (size_t)n_geom * ((n_t + GS_THREADS - 1) / GS_THREADS);
    if (zi) {
        st = launch_zi(A, atab, n_in, n_edge, smem, max_items, s);
    } else {
        cudaError_t e = cudaStreamWaitEvent(s, plan->ev_join, 0);
        if (e != cudaSuccess) return set_cuda_error(e, "pt_gimenez join");
        st = launch_cheb_eval(A, dtab, max_items, plan->ev0, plan->ev1, s);
    }
    if (st) return st;
    if (ssr) st = launch_ssr_rows(A.flux, y, wt, n_t, n_b, (size_t)orb->n_v * n_b, (float *)(wb + L.part), ssr, s);
    return st;
}

extern "C" {

int pt_gimenez(pt_gim_plan plan, const double *t, int n_t, const pt_orbit *orb, const float *k, int k_per_band,
               const float *ld, int n_b, int n_ss, double t_exp, int max_iter, const float *y, const float *wt,
               float *flux, float *ssr, void *work, size_t work_bytes, int *n_bad, pt_stream_t stream)
{
    return gimenez_impl(plan, 0, 0, t, n_t, orb, k, k_per_band, ld, n_b, n_ss, t_exp, max_iter, y, wt, flux, ssr,
                        work, work_bytes, n_bad, stream);
}

size_t pt_gimenez_zi_work_bytes(pt_gim_plan plan, int n_in, int n_edge, int n_t, int n_v, int n_b, int k_per_band)
{
    if (!plan || n_t < 0 || n_v < 0 || n_b < 1 || n_in < 2 || n_edge < 1) return 0;
    return work_layout(n_t, n_v, n_b, k_per_band, plan->N + 1, plan->n_j, n_in + n_edge).total;
}

int pt_gimenez_zi(pt_gim_plan plan, int n_in, int n_edge, const double *t, int n_t, const pt_orbit *orb,
                  const float *k, int k_per_band, const float *ld, int n_b, int n_ss, double t_exp, int max_iter,
                  const float *y, const float *wt, float *flux, float *ssr, void *work, size_t work_bytes,
                  int *n_bad, pt_stream_t stream)
{
    if (n_in < 2) return PT_ERR_ARG;
    return gimenez_impl(plan, n_in, n_edge, t, n_t, orb, k, k_per_band, ld, n_b, n_ss, t_exp, max_iter, y, wt, flux,
                        ssr, work, work_bytes, n_bad, stream);
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
    // the tile kernel: its scratch is small (records, time split, partials)
    size_t need = work_layout(n_t, orb->n_v, n_b, k_per_band, 0, 0).total;
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
    return ma_quad_impl(nullptr, t, n_t, orb, k, k_per_band, ld, n_b, n_ss, t_exp, max_iter, y, wt, flux, ssr,
                        scratch, (size_t)PT_MA_NOALLOC_SCRATCH_BYTES, n_bad, stream);
}
