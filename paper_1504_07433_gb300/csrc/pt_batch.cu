// pt_batch.cu -- one persistent, graph-captured launch over many MCMC walkers,
// passbands and light curves of uneven length (spectrophotometry: the paper's
// motivation in Sec. 1; per-passband radius ratios and limb darkening,
// Secs. 2.2.2 and 3.5; the device-side likelihood of Sec. 3.4).
//
// Work list: (walker, time tile) items, tiles never straddle a light curve,
// ordered tile-major so that consecutive items share their times and
// observations in L2.  A grid of (SMs x CTAs/SM) persistent CTAs pulls items
// through an atomic counter.  Per item:
//   A. one thread per time: phase reduction, window test (largest k of the
//      walker's passbands), z for in-window times, compaction;
//   B. (in-window time, passband) units on full warps: Mandel-Agol terms with
//      the passband's own k, limb darkening with its own (u1, u2);
//   C. one warp per passband: coalesced flux stores, residual sums reduced in
//      a fixed order into per-(walker, passband, tile) partials.
// The plan autotunes the tile length and the CTAs per SM by timing the
// candidates on the caller's buffers, then captures counter reset + set-up +
// persistent kernel + residual reduction into one CUDA graph.
#include <cuda_runtime.h>

#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "../../include/pt.h"
#include "pt_device.cuh"

using pt::GeomRec;

namespace pt_internal {
int set_error(int status, const char *where, const char *msg);   // pt_lc.cu
bool ma_table_view(pt_ma_table t, const float4 **tab, int *n_k, int *n_z, float *k_lo, float *k_hi, float *inv_dk,
                   float *inv_dz);                                   // pt_lc.cu
}

namespace {

struct BatchItem {
    int v, start, len, tile;
};

struct BatchArgs {
    const float2 *tsplit;
    int n_t;
    const GeomRec *rec;
    const float *k;      // [n_v][n_b]
    const float *ld;     // [n_v][n_b][2]
    int n_v, n_b, n_ss;
    float t_exp;
    int max_iter;
    const float *y, *wt; // [n_b][n_t]
    float *flux;         // [n_v][n_b][n_t]
    float *ssr_part;     // [n_v][n_b][n_tiles]
    int n_tiles;
    const BatchItem *items;
    int n_items;
    int *counter;
    int *n_bad;
    int khat;            // k_mode 1: terms once per time with k_hat (Sec. 3.5)
    // k_mode 2: the Mandel-Agol terms interpolated from this table (Sec. 2.2.3)
    const float4 *mtab;
    int mn_k, mn_z;
    float mk_lo, mk_hi, minv_dk, minv_dz;
};

struct BatchSetupArgs {
    const double *t;
    int n_t;
    float2 *tsplit;
    pt_orbit orb;
    const float *k;
    int n_b;
    float half_exp;
    GeomRec *rec;
    int n_vblocks;
    int khat;
};

__global__ void batch_setup_kernel(BatchSetupArgs s)
{
    if ((int)blockIdx.x < s.n_vblocks) {
        int v = blockIdx.x * blockDim.x + threadIdx.x;
        if (v >= s.orb.n_v) return;
        // the geometry's k: the largest passband k (its window covers every
        // passband), or in k_hat mode the mean, the only k evaluated
        float kmax = 0.0f, ksum = 0.0f;
        for (int b = 0; b < s.n_b; ++b) {
            float kb = s.k[(size_t)v * s.n_b + b];
            kmax = fmaxf(kmax, kb);
            ksum += kb;
        }
        if (s.khat) kmax = ksum / (float)s.n_b;
        bool ecc = s.orb.e != nullptr;
        pt::make_geom_rec(s.orb.t0[v], s.orb.P[v], s.orb.a[v], s.orb.inc[v], ecc, ecc ? s.orb.e[v] : 0.0f,
                          ecc ? s.orb.w[v] : 0.0f, kmax, s.half_exp, &s.rec[v]);
    } else {
        int i = (blockIdx.x - s.n_vblocks) * blockDim.x + threadIdx.x;
        if (i < s.n_t) {
            double x = s.t[i];
            float h = (float)x;
            s.tsplit[i] = make_float2(h, (float)(x - (double)h));
        }
    }
}

template <int TT, bool INTERP>
__global__ void __launch_bounds__(TT) batch_kernel(BatchArgs A)
{
    extern __shared__ __align__(16) float dyn[];
    float *fbuf = dyn;                    // [n_b][TT]
    float *swt = dyn + A.n_b * TT;        // [n_b][4]: we, wd, wn, k (k_hat mode: k^2 / k_hat^2)
    __shared__ GeomRec srec;
    __shared__ float sdt[TT], sz[TT];
    __shared__ float ste[3][TT];          // k_hat mode: supersample-mean terms per time
    __shared__ unsigned char sflag[TT];
    __shared__ unsigned short squeue[TT];
    __shared__ int sqn, s_item, sbad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = TT / 32;
    if (tid == 0) sbad = 0;
    bool bad = false;
    for (;;) {
        if (tid == 0) {
            s_item = atomicAdd(A.counter, 1);
            sqn = 0;
        }
        __syncthreads();
        const int it = s_item;
        if (it >= A.n_items) break;
        const BatchItem item = A.items[it];
        const int v = item.v;
        if (tid < 6)
            reinterpret_cast<float4 *>(&srec)[tid] = reinterpret_cast<const float4 *>(&A.rec[v])[tid];
        for (int b = tid; b < A.n_b; b += TT) {
            float we, wd, wn;
            pt::ma_weights(A.ld[((size_t)v * A.n_b + b) * 2], A.ld[((size_t)v * A.n_b + b) * 2 + 1], &we, &wd, &wn);
            swt[4 * b] = we;
            swt[4 * b + 1] = wd;
            swt[4 * b + 2] = wn;
            float kb = A.k[(size_t)v * A.n_b + b];
            if (A.khat) {
                float r = kb / A.rec[v].k;
                kb = r * r;
            }
            swt[4 * b + 3] = kb;
        }
        __syncthreads();
        // A: window test, z, compaction
        bool inw = false;
        float dt = 0.0f, z = PT_ZBEHIND;
        if (tid < item.len) {
            float2 ts = A.tsplit[item.start + tid];
            if (pt::maybe_in_window(ts.x, srec)) {
                dt = pt::reduce_time(ts.x, ts.y, srec);
                inw = dt >= srec.win_lo && dt <= srec.win_hi;
            }
            if (inw && A.n_ss == 1) z = pt::orbit_z<true>(srec, dt, A.max_iter, &bad);
        }
        sdt[tid] = dt;
        sz[tid] = z;
        sflag[tid] = inw ? 1 : 0;
        int slot = pt::warp_append(&sqn, inw);
        if (inw) squeue[slot] = (unsigned short)tid;
        __syncthreads();
        // B: (time, passband) units
        const int nq = sqn;
        const int nu = nq * A.n_b;
        const float inv_ss = 1.0f / (float)A.n_ss;
        if (A.khat) {
            // the terms once per in-window time, with k_hat ...
            for (int qi = tid; qi < nq; qi += TT) {
                int tl = squeue[qi];
                float le = 0.0f, ld = 0.0f, ed = 0.0f;
                float warm[3] = {__int_as_float(0x7fffffff), 0.0f, 0.0f};   // Kepler warm start (none yet)
                for (int s = 0; s < A.n_ss; ++s) {
                    float zs = sz[tl];
                    if (A.n_ss > 1) {
                        float dts = sdt[tl] + A.t_exp * (((float)s + 0.5f) * inv_ss - 0.5f);
                        zs = pt::orbit_z<true>(srec, dts, A.max_iter, &bad, warm);
                    }
                    float a0, a1, a2;
                    pt::ma_terms(srec.k, zs, &a0, &a1, &a2);
                    le += a0;
                    ld += a1;
                    ed += a2;
                }
                ste[0][tl] = le * inv_ss;
                ste[1][tl] = ld * inv_ss;
                ste[2][tl] = ed * inv_ss;
            }
            __syncthreads();
            // ... then each passband's depth scaled by k_b^2 / k_hat^2
            for (int u = tid; u < nu; u += TT) {
                int b = u / nq, qi = u - b * nq;
                int tl = squeue[qi];
                float dep = swt[4 * b] * ste[0][tl] + swt[4 * b + 1] * ste[1][tl] + swt[4 * b + 2] * ste[2][tl];
                fbuf[b * TT + tl] = 1.0f - swt[4 * b + 3] * dep;
            }
        }
        // unit u = b nq + qi; the thread's units advance by TT = dq nq + dr
        const int dq = nq > 0 ? TT / nq : 0, dr = nq > 0 ? TT - dq * nq : 0;
        int ub = nq > 0 ? tid / nq : 0, uq = tid - ub * nq;
        for (int u = A.khat ? nu : tid; u < nu; u += TT) {
            const int b = ub, qi = uq;
            ub += dq;
            uq += dr;
            if (uq >= nq) {
                uq -= nq;
                ++ub;
            }
            int tl = squeue[qi];
            float kb = swt[4 * b + 3];
            float le, ld, ed;
            if (A.n_ss == 1) {
                if (INTERP)
                    pt::ma_interp(A.mtab, A.mn_k, A.mn_z, A.mk_lo, A.mk_hi, A.minv_dk, A.minv_dz, kb, sz[tl], &le, &ld, &ed);
                else
                    pt::ma_terms(kb, sz[tl], &le, &ld, &ed);
            } else {
                le = ld = ed = 0.0f;
                float warm[3] = {__int_as_float(0x7fffffff), 0.0f, 0.0f};   // Kepler warm start (none yet)
                for (int s = 0; s < A.n_ss; ++s) {
                    float dts = sdt[tl] + A.t_exp * (((float)s + 0.5f) * inv_ss - 0.5f);
                    float zs = pt::orbit_z<true>(srec, dts, A.max_iter, &bad, warm);
                    float a0, a1, a2;
                    if (INTERP)
                        pt::ma_interp(A.mtab, A.mn_k, A.mn_z, A.mk_lo, A.mk_hi, A.minv_dk, A.minv_dz, kb, zs, &a0, &a1, &a2);
                    else
                        pt::ma_terms(kb, zs, &a0, &a1, &a2);
                    le += a0;
                    ld += a1;
                    ed += a2;
                }
                le *= inv_ss;
                ld *= inv_ss;
                ed *= inv_ss;
            }
            fbuf[b * TT + tl] = 1.0f - (swt[4 * b] * le + swt[4 * b + 1] * ld + swt[4 * b + 2] * ed);
        }
        __syncthreads();
        // C: one warp per passband
        for (int b = warp; b < A.n_b; b += NW) {
            float acc = 0.0f;
            const size_t row = (size_t)v * A.n_b + b;
            for (int t = lane; t < item.len; t += 32) {
                float f = sflag[t] ? fbuf[b * TT + t] : 1.0f;
                int i = item.start + t;
                if (A.flux) A.flux[row * A.n_t + i] = f;
                if (A.ssr_part) {
                    float r = A.y[(size_t)b * A.n_t + i] - f;
                    acc = fmaf((A.wt ? A.wt[(size_t)b * A.n_t + i] : 1.0f) * r, r, acc);
                }
            }
            if (A.ssr_part) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0) A.ssr_part[row * A.n_tiles + item.tile] = acc;
            }
        }
        __syncthreads();
    }
    if (bad) atomicAdd(&sbad, 1);
    __syncthreads();
    if (tid == 0 && sbad && A.n_bad) atomicAdd(A.n_bad, sbad);
}

__global__ void batch_reduce_kernel(const float *part, int rows, int n_tiles, float *ssr)
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

size_t dyn_smem(int TT, int n_b) { return (size_t)n_b * TT * sizeof(float) + (size_t)n_b * 4 * sizeof(float); }

}  // namespace

struct pt_batch_plan_s {
    pt_batch_desc d;
    int tt, ctas_per_sm, grid, n_sm;
    int n_items, n_tiles;
    BatchItem *d_items;
    int *d_counter;
    GeomRec *d_rec;
    float2 *d_tsplit;
    float *d_part;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    float tuned_ms;
    std::vector<int> h_offsets;
};

namespace {

int berr(cudaError_t e, const char *where)
{
    return pt_internal::set_error(PT_ERR_CUDA, where, cudaGetErrorString(e));
}

// Tiles of length tt within each light curve; items tile-major.
void build_items(const pt_batch_plan_s &p, int tt, std::vector<BatchItem> *items, int *n_tiles)
{
    std::vector<std::pair<int, int>> tiles;
    for (size_t j = 0; j + 1 < p.h_offsets.size(); ++j)
        for (int s = p.h_offsets[j]; s < p.h_offsets[j + 1]; s += tt)
            tiles.push_back({s, std::min(tt, p.h_offsets[j + 1] - s)});
    *n_tiles = (int)tiles.size();
    items->clear();
    items->reserve((size_t)tiles.size() * p.d.orb.n_v);
    for (size_t q = 0; q < tiles.size(); ++q)
        for (int v = 0; v < p.d.orb.n_v; ++v) items->push_back({v, tiles[q].first, tiles[q].second, (int)q});
}

template <int TT>
int launch_batch_tt(const BatchArgs &A, int grid, size_t smem, cudaStream_t s)
{
    if (A.mtab)
        batch_kernel<TT, true><<<grid, TT, smem, s>>>(A);
    else
        batch_kernel<TT, false><<<grid, TT, smem, s>>>(A);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PT_OK : berr(e, "batch_kernel");
}

template <bool I>
cudaError_t set_smem_attr_i(int tt, size_t smem)
{
    cudaError_t e = cudaSuccess;
    if (tt == 64) e = cudaFuncSetAttribute(batch_kernel<64, I>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (tt == 128) e = cudaFuncSetAttribute(batch_kernel<128, I>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (tt == 256) e = cudaFuncSetAttribute(batch_kernel<256, I>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
}

int set_smem_attr(int tt, size_t smem, bool interp)
{
    cudaError_t e = interp ? set_smem_attr_i<true>(tt, smem) : set_smem_attr_i<false>(tt, smem);
    return e == cudaSuccess ? PT_OK : berr(e, "cudaFuncSetAttribute");
}

template <bool I>
int max_ctas_per_sm_i(int tt, size_t smem)
{
    int n = 0;
    if (tt == 64) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<64, I>, tt, smem);
    if (tt == 128) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<128, I>, tt, smem);
    if (tt == 256) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<256, I>, tt, smem);
    return n;
}

int max_ctas_per_sm(int tt, size_t smem, bool interp)
{
    return interp ? max_ctas_per_sm_i<true>(tt, smem) : max_ctas_per_sm_i<false>(tt, smem);
}

// Enqueue one full evaluation (counter reset, set-up, persistent kernel,
// residual reduction) for the plan's current configuration.
int enqueue(pt_batch_plan_s &p, cudaStream_t s)
{
    const pt_batch_desc &d = p.d;
    cudaError_t e = cudaMemsetAsync(p.d_counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return berr(e, "cudaMemsetAsync");
    BatchSetupArgs sa;
    sa.t = d.t;
    sa.n_t = d.n_t;
    sa.tsplit = p.d_tsplit;
    sa.orb = d.orb;
    sa.k = d.k;
    sa.khat = d.k_mode == 1;
    sa.n_b = d.n_b;
    sa.half_exp = (float)(0.5 * d.t_exp);
    sa.rec = p.d_rec;
    sa.n_vblocks = (d.orb.n_v + 63) / 64;
    batch_setup_kernel<<<sa.n_vblocks + (d.n_t + 63) / 64, 64, 0, s>>>(sa);
    e = cudaGetLastError();
    if (e != cudaSuccess) return berr(e, "batch_setup_kernel");
    BatchArgs A;
    A.tsplit = p.d_tsplit;
    A.n_t = d.n_t;
    A.rec = p.d_rec;
    A.k = d.k;
    A.khat = d.k_mode == 1;
    A.mtab = nullptr;
    A.mn_k = A.mn_z = 0;
    A.mk_lo = A.mk_hi = A.minv_dk = A.minv_dz = 0.0f;
    if (d.k_mode == 2 && !pt_internal::ma_table_view(d.table, &A.mtab, &A.mn_k, &A.mn_z, &A.mk_lo, &A.mk_hi,
                                                     &A.minv_dk, &A.minv_dz))
        return pt_internal::set_error(PT_ERR_ARG, "pt_batch_run", "k_mode 2 needs an interpolation table");
    A.ld = d.ld;
    A.n_v = d.orb.n_v;
    A.n_b = d.n_b;
    A.n_ss = d.n_ss;
    A.t_exp = (float)d.t_exp;
    A.max_iter = d.max_iter;
    A.y = d.y;
    A.wt = d.wt;
    A.flux = d.flux;
    A.ssr_part = d.ssr ? p.d_part : nullptr;
    A.n_tiles = p.n_tiles;
    A.items = p.d_items;
    A.n_items = p.n_items;
    A.counter = p.d_counter;
    A.n_bad = d.n_bad;
    size_t smem = dyn_smem(p.tt, d.n_b);
    int st = PT_OK;
    if (p.tt == 64) st = launch_batch_tt<64>(A, p.grid, smem, s);
    if (p.tt == 128) st = launch_batch_tt<128>(A, p.grid, smem, s);
    if (p.tt == 256) st = launch_batch_tt<256>(A, p.grid, smem, s);
    if (st) return st;
    if (d.ssr) {
        int rows = d.orb.n_v * d.n_b;
        batch_reduce_kernel<<<(rows * 32 + 255) / 256, 256, 0, s>>>(p.d_part, rows, p.n_tiles, d.ssr);
        e = cudaGetLastError();
        if (e != cudaSuccess) return berr(e, "batch_reduce_kernel");
    }
    return PT_OK;
}

int configure(pt_batch_plan_s &p, int tt, int cps)
{
    std::vector<BatchItem> items;
    int n_tiles = 0;
    build_items(p, tt, &items, &n_tiles);
    cudaFree(p.d_items);
    cudaFree(p.d_part);
    p.d_items = nullptr;
    p.d_part = nullptr;
    cudaError_t e = cudaMalloc(&p.d_items, std::max<size_t>(1, items.size()) * sizeof(BatchItem));
    if (e != cudaSuccess) return berr(e, "cudaMalloc items");
    e = cudaMemcpy(p.d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return berr(e, "cudaMemcpy items");
    if (p.d.ssr) {
        e = cudaMalloc(&p.d_part, (size_t)p.d.orb.n_v * p.d.n_b * n_tiles * sizeof(float));
        if (e != cudaSuccess) return berr(e, "cudaMalloc partials");
    }
    p.tt = tt;
    p.ctas_per_sm = cps;
    p.grid = cps * p.n_sm;
    p.n_items = (int)items.size();
    p.n_tiles = n_tiles;
    return set_smem_attr(tt, dyn_smem(tt, p.d.n_b), p.d.k_mode == 2);
}

void free_plan(pt_batch_plan_s *p)
{
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    cudaFree(p->d_items);
    cudaFree(p->d_counter);
    cudaFree(p->d_rec);
    cudaFree(p->d_tsplit);
    cudaFree(p->d_part);
    delete p;
}

}  // namespace

extern "C" {

int pt_batch_plan_create(const pt_batch_desc *d, int autotune, pt_batch_plan *out)
{
    if (!d || !out) return PT_ERR_ARG;
    *out = nullptr;
    const pt_orbit &o = d->orb;
    if (o.n_v < 1 || d->n_t < 1 || d->n_lc < 1 || d->n_b < 1 || d->n_b > 256 || d->n_ss < 1 || d->n_ss > 256 ||
        d->max_iter < 1 || d->max_iter > 64)
        return PT_ERR_ARG;
    if (!d->t || !d->lc_offsets || !o.t0 || !o.P || !o.a || !o.inc || !d->k || !d->ld) return PT_ERR_ARG;
    if ((o.e == nullptr) != (o.w == nullptr)) return PT_ERR_ARG;
    if (!d->flux && !d->ssr) return PT_ERR_ARG;
    if (d->k_mode < 0 || d->k_mode > 2) return PT_ERR_ARG;
    if ((d->k_mode == 2) != (d->table != nullptr)) return PT_ERR_ARG;
    if (d->ssr && !d->y) return PT_ERR_ARG;
    if (!(d->t_exp >= 0.0 && d->t_exp < 1.0e30))
        return pt_internal::set_error(PT_ERR_DOMAIN, "pt_batch_plan_create", "exposure time must be finite and >= 0");
    if (d->lc_offsets[0] != 0 || d->lc_offsets[d->n_lc] != d->n_t) return PT_ERR_ARG;
    for (int j = 0; j < d->n_lc; ++j)
        if (d->lc_offsets[j + 1] < d->lc_offsets[j]) return PT_ERR_ARG;
    pt_batch_plan_s *p = new pt_batch_plan_s();
    p->d = *d;
    p->h_offsets.assign(d->lc_offsets, d->lc_offsets + d->n_lc + 1);
    p->d.lc_offsets = nullptr;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaMalloc(&p->d_counter, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_rec, (size_t)o.n_v * sizeof(GeomRec));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_tsplit, (size_t)d->n_t * sizeof(float2));
    if (e != cudaSuccess) {
        int st = berr(e, "pt_batch_plan_create");
        free_plan(p);
        return st;
    }
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        int st = berr(e, "cudaStreamCreate");
        free_plan(p);
        return st;
    }
    // autotuner: tile length x CTAs per SM, timed on the caller's buffers
    int best_tt = 128, best_cps = 0;
    float best = 1e30f;
    const int tts[3] = {64, 128, 256};
    int st = PT_OK;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int ti = 0; ti < 3 && st == PT_OK; ++ti) {
        int tt = tts[ti];
        if (!autotune && tt != 128) continue;
        size_t smem = dyn_smem(tt, d->n_b);
        if (smem > 200 * 1024) continue;
        st = set_smem_attr(tt, smem, d->k_mode == 2);
        if (st) break;
        int mx = max_ctas_per_sm(tt, smem, d->k_mode == 2);
        if (mx < 1) continue;
        int cands[4] = {mx, mx / 2, mx / 4, 1};
        for (int ci = 0; ci < 4 && st == PT_OK; ++ci) {
            int cps = cands[ci];
            if (cps < 1 || (ci > 0 && cps == cands[ci - 1])) continue;
            if (!autotune && ci > 0) break;
            st = configure(*p, tt, cps);
            if (st) break;
            st = enqueue(*p, cs);   // warm-up
            if (st) break;
            float ms_tot = 0.0f;
            const int reps = autotune ? 2 : 1;
            for (int r = 0; r < reps && st == PT_OK; ++r) {
                cudaEventRecord(e0, cs);
                st = enqueue(*p, cs);
                cudaEventRecord(e1, cs);
                cudaEventSynchronize(e1);
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms_tot += ms;
            }
            float ms = ms_tot / reps;
            if (st == PT_OK && ms < best) {
                best = ms;
                best_tt = tt;
                best_cps = cps;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == PT_OK && best_cps == 0) st = PT_ERR_ARG;
    if (st == PT_OK) st = configure(*p, best_tt, best_cps);
    if (st == PT_OK) {
        e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) st = berr(e, "autotune");
    }
    p->tuned_ms = best;
    // capture the evaluation into a graph
    if (st == PT_OK) {
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) st = berr(e, "cudaStreamBeginCapture");
        if (st == PT_OK) {
            int st2 = enqueue(*p, cs);
            e = cudaStreamEndCapture(cs, &p->graph);
            if (st2) st = st2;
            else if (e != cudaSuccess) st = berr(e, "cudaStreamEndCapture");
        }
        if (st == PT_OK) {
            e = cudaGraphInstantiate(&p->exec, p->graph, 0);
            if (e != cudaSuccess) st = berr(e, "cudaGraphInstantiate");
        }
    }
    cudaStreamDestroy(cs);
    if (st) {
        free_plan(p);
        return st;
    }
    *out = p;
    return PT_OK;
}

int pt_batch_run(pt_batch_plan p, pt_stream_t stream)
{
    if (!p || !p->exec) return PT_ERR_ARG;
    cudaError_t e = cudaGraphLaunch(p->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? PT_OK : berr(e, "cudaGraphLaunch");
}

int pt_batch_plan_info(pt_batch_plan p, int *tile, int *ctas_per_sm, int *n_items, float *tuned_ms)
{
    if (!p) return PT_ERR_ARG;
    if (tile) *tile = p->tt;
    if (ctas_per_sm) *ctas_per_sm = p->ctas_per_sm;
    if (n_items) *n_items = p->n_items;
    if (tuned_ms) *tuned_ms = p->tuned_ms;
    return PT_OK;
}

int pt_batch_plan_destroy(pt_batch_plan p)
{
    free_plan(p);
    return PT_OK;
}

}  // extern "C"
