// Applying the compressed view-factor matrix (Algorithm 5) and the Jacobi
// solve of B = E + diag(rho) F B (Sections 3, 5.1).
//
// Layout: everything runs in tree order.  X and Y (and E, B) are permuted
// once per call; every block's rows and columns are then contiguous ranges
// (dense, CSR) or sorted index lists (SVD).
//
// Per multiply:
//   phase 1  T_b = V'_b^T X[cols_b]      for each SVD block (q x R), split in
//            row chunks of V' whose partial sums the last chunk to finish
//            adds in chunk order (deterministic, no float atomics);
//   phase 2  one CTA per row tile (a tree leaf, <= 64 rows) and RHS panel:
//            every block crossing the tile adds its rows (dense rows, CSR
//            rows, or U'_b T_b); each row is owned by one warp and kept in
//            registers, so Y is written once, in a fixed order.
// The Jacobi update, the per-column residual partials and (for refinement)
// the FP64-accumulated residual are fused into the phase-2 epilogue.
#include <cuda/atomic>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <memory>
#include <mutex>
#include <queue>

#include "vf_bulk.cuh"
#include "vf_hmat.cuh"
#include "vf_tensor.cuh"

namespace vf {

constexpr int kTileRows = 64;
constexpr int kWarps = 8;


struct ApplyArgs {
    const int32_t* tile_first;
    const int32_t* tile_count;
    const int32_t* tile_page_ptr;  // per (tile, warp): first page; ntiles * kWarps + 1 entries
    const int32_t* tile_order;
    int64_t nparts;                // phase-1 partial floats per RHS column (units of cut blocks, q each)
    int64_t n;                     // facets
    int64_t nT;                    // T slots per RHS column
    int R;                         // total RHS columns
};

// Both phases stream the matrix as pages (see vf_hmat.cuh) through per-warp
// prefetch pipelines: lane 0 of each warp issues one bulk asynchronous copy
// per page into one of kStages shared-memory stages (an mbarrier per stage
// tracks the bytes) while the warp computes on a page that has arrived.  On
// arrival the warp gathers every x (or T) value the page's records need in
// one round, in place over the page's x list, so the records then compute
// from shared memory only.  Few, large copies in flight per SM (kStages x
// warps x CTAs ~ 48 of 4 KB) keep HBM streaming efficiently.  Every sum has
// one owner and one order, so results are bit-reproducible with no float
// atomics:
//  * dense and SVD slabs (column-major): lane r owns slab row r (and r + 32);
//  * CSR rows: lane r walks row r's nonzeros; a long row is split across
//    lanes and reduced by a fixed butterfly;
//  * phase-1 V' rows: a group of g = pow2ceil(min(q, 32)) lanes per row,
//    lane (sub, k) accumulates column k over its rows, groups added by a
//    fixed butterfly.
// Row sums go to per-warp row slots in shared memory; the CTA adds the
// warps' slots in warp order.  Every wait is bounded, and a warp that stops
// early first waits (bounded) for its own copies in flight.
#ifndef VF_STAGES
#define VF_STAGES 2
#endif
constexpr int kStages = VF_STAGES;
constexpr uint32_t kWaitLimit = 1u << 22;  // polls before a wait reports a timeout (the default)
// The page waits of the multiply kernels poll at most g_wait_polls times
// (vf_set_wait_limit; read by each kernel at its start, so solve graphs see
// changes too).  The drain before an early exit always uses kWaitLimit, so a
// short limit never lets a warp leave with bulk copies in flight.
__device__ uint32_t g_wait_polls = kWaitLimit;

template <class T> __device__ __forceinline__ float lds(const T* p);
template <> __device__ __forceinline__ float lds<float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float lds<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }
template <> __device__ __forceinline__ float lds<__nv_fp8_e4m3>(const __nv_fp8_e4m3* p) { return float(*p); }

struct WarpPipe {
    uint64_t bar[kStages];
    __align__(16) unsigned char buf[kStages][kPage];
};

struct PageArgs {
    const unsigned char* pages;
    const uint16_t* used;
};

__device__ __forceinline__ void issue_page(const PageArgs& pg, int64_t page, WarpPipe& wp, int s) {
    const uint32_t bytes = ((uint32_t)pg.used[page] + 15u) & ~15u;
    mbar_arrive_expect_tx(&wp.bar[s], bytes);
    bulk_g2s(wp.buf[s], pg.pages + page * (int64_t)kPage, bytes, &wp.bar[s]);
}

__device__ __forceinline__ void pipe_init(WarpPipe& wp) {
    for (int s = 0; s < kStages; ++s) mbar_init(&wp.bar[s], 1);
    mbar_init_fence();
}

// Wait (bounded) for the copies this warp issued but did not consume, so a
// warp that stops early never leaves bulk copies in flight into its stages.
__device__ __forceinline__ void drain(WarpPipe& wp, int consumed, int issued) {
    for (int j = consumed; j < issued; ++j) mbar_wait(&wp.bar[j % kStages], (uint32_t)((j / kStages) & 1), kWaitLimit);
}

// x source of entry v of a page's x list for RHS column c of the panel
__device__ __forceinline__ float x_of(const ApplyArgs& a, const float* X, const float* Tp, int32_t v, int c) {
    return v >= 0 ? __ldg(X + (int64_t)c * a.n + v) : Tp[(int64_t)c * a.nT + (-1 - v)];
}

// Panel column c of the x entries of a page, entry e = lane + 32 j in v[j]:
// all loads issued before any is used.
__device__ __forceinline__ void load_col(const ApplyArgs& a, const float* X, const float* Tp, const int32_t* xl,
                                         int nx, int c, float (&v)[kXMax / 32]) {
    const int lane = threadIdx.x & 31;
    const int nj = (nx + 31) >> 5;  // warp-uniform: rounds past it are skipped
#pragma unroll
    for (int j = 0; j < kXMax / 32; ++j) {
        if (j < nj) {
            const int e = lane + 32 * j;
            v[j] = e < nx ? x_of(a, X, Tp, xl[e], c) : 0.f;
        }
    }
}

__device__ __forceinline__ void store_col(int nx, const float (&v)[kXMax / 32], float* xv) {
    const int lane = threadIdx.x & 31;
    const int nj = (nx + 31) >> 5;
#pragma unroll
    for (int j = 0; j < kXMax / 32; ++j) {
        if (j < nj) {
            const int e = lane + 32 * j;
            if (e < nx) xv[e] = v[j];
        }
    }
}

// Single column: gather the page's x list in place (each lane overwrites the
// entries it read), so the records then read x values from the page itself.
__device__ __forceinline__ void gather_in_place(const ApplyArgs& a, const float* X, const float* Tp,
                                                unsigned char* page) {
    const int nx = (int)reinterpret_cast<const uint32_t*>(page)[2];
    int32_t* xl = reinterpret_cast<int32_t*>(page + kPageHdr);
    float v[kXMax / 32];
    load_col(a, X, Tp, xl, nx, 0, v);
    store_col(nx, v, reinterpret_cast<float*>(xl));
    __syncwarp();
}

// ------------------------------------------------------------ phase 1
// T_b = V'_b^T X[cols_b] from phase-1 records, one panel column at a time
// (xv: that column's x values, indexed by x-list entry).  T: per panel
// RB x nT (column c at c * nT).  A block whose V' rows span several records
// (chunks) has them in one warp, in order: the warp carries the running
// sum in shared memory (carry[c * 128 + k]) and writes T after the last
// chunk.  A very large block is cut into several such units; each unit then
// writes its sum to a partial slot and k_p1_reduce adds the units in order.
template <class T, int RB>
__device__ __forceinline__ void p1_column(const ApplyArgs& a, const float* xv, const unsigned char* rec, int c,
                                          float* __restrict__ Tbuf, float* __restrict__ part,
                                          float* __restrict__ carry, int panel) {
    const int lane = threadIdx.x & 31;
    const uint4 h0 = reinterpret_cast<const uint4*>(rec)[0], h1 = reinterpret_cast<const uint4*>(rec)[1];
    const int nrows = (int)((h0.x >> 8) & 0xffu), q = (int)h0.y, xb = (int)h0.z;
    const float sc = __uint_as_float(h0.w);
    const int chunk = (int)h1.x, nch = (int)h1.y, slot = (int)h1.z, offT = (int)h1.w;
    const T* sV = reinterpret_cast<const T*>(rec + kP1Hdr);
    const int lg = q >= 32 ? 5 : (q <= 1 ? 0 : 32 - __clz(q - 1));  // g = 2^lg lanes per row
    const int g = 1 << lg;
    const int step = 32 >> lg;
    const int sub = lane >> lg, kk = lane & (g - 1);
    const int nk = (q + 31) >> 5;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    if (q <= 32) {
        if (kk < q)
#pragma unroll 4
            for (int j = sub; j < nrows; j += step) acc[0] = fmaf(lds(sV + j * q + kk), xv[xb + j], acc[0]);
        for (int o = 16; o >= g; o >>= 1) acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], o);
    } else {
        for (int j = 0; j < nrows; ++j) {  // q > 32: the whole warp shares each row
            const float x = xv[xb + j];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int k = lane + 32 * t;
                if (t < nk && k < q) acc[t] = fmaf(lds(sV + j * q + k), x, acc[t]);
            }
        }
        // g = 32: the warp is one group, nothing to add across lanes
    }
    if (sub != 0) return;
    // the unit's result goes to T (scaled) or, for a unit of a cut block, to its partial slot
    float* dst = slot < 0 ? Tbuf + ((int64_t)panel * RB + c) * a.nT + offT
                          : part + ((int64_t)panel * RB + c) * a.nparts + slot;
    const float f = slot < 0 ? sc : 1.f;
    float* cr = carry + c * 128;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int k = kk + 32 * t;
        if (t < nk && k < q) {
            const float v = chunk == 0 ? acc[t] : cr[k] + acc[t];
            if (chunk == nch - 1) dst[k] = v * f;
            else cr[k] = v;
        }
    }
}

// T of the blocks cut into several units: the unit sums added in unit
// order, then scaled.  One warp per (cut block, panel); split[5 i ..] =
// offset of the block's partials (unit u at offset + u q in each column's
// partial area), units, q, T slot, block.
template <int RB>
__global__ void __launch_bounds__(256) k_p1_reduce(ApplyArgs a, const int32_t* __restrict__ split, int64_t nsplit,
                                                   const float* __restrict__ scales, const float* __restrict__ part,
                                                   float* __restrict__ Tbuf) {
    const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= nsplit) return;
    const int32_t* d = split + 5 * i;
    const int first = d[0], nch = d[1], q = d[2], offT = d[3];
    const float sc = scales ? scales[d[4]] : 1.f;
    const int panel = blockIdx.y;
    for (int c = 0; c < RB && panel * RB + c < a.R; ++c)
        for (int k = lane; k < q; k += 32) {
            const float* pb = part + ((int64_t)panel * RB + c) * a.nparts + first;
            float sum = 0.f;
            for (int cc = 0; cc < nch; ++cc) sum += pb[cc * q + k];
            Tbuf[((int64_t)panel * RB + c) * a.nT + offT + k] = sum * sc;
        }
}

// Walk a page's records (after its header and x list); f(record) returns
// nothing, the record sizes come from the headers.
template <class T, class F>
__device__ __forceinline__ void for_records(const unsigned char* page, F f) {
    const uint32_t* ph = reinterpret_cast<const uint32_t*>(page);
    const int nrec = (int)ph[0];
    uint32_t off = page_rec0(ph[2]);
    for (int r = 0; r < nrec; ++r) {
        const uint2 h = *reinterpret_cast<const uint2*>(page + off);
        const int kind = (int)(h.x & 0xffu), cnt = (int)((h.x >> 8) & 0xffu);
        f(page + off);
        off += rec_bytes(kind, cnt, (int)h.y, (int)sizeof(T));
    }
}

// Per-warp x buffers for panels of more than one column: two columns, so
// the loads of column c + 1 are in flight while column c computes.
struct XBuf {
    float v[2][kXMax];
};

// Every panel column of one page: f(xv, c) computes column c from xv.  One
// column gathers in place; more columns go through the warp's XBuf.
template <int RB, class F>
__device__ __forceinline__ void page_columns(const ApplyArgs& a, const float* X, const float* Tp, unsigned char* page,
                                             XBuf* xb, int p0, F f) {
    if (RB == 1) {
        gather_in_place(a, X, Tp, page);
        f(reinterpret_cast<const float*>(page + kPageHdr), 0);
        return;
    }
    const int nx = (int)reinterpret_cast<const uint32_t*>(page)[2];
    const int32_t* xl = reinterpret_cast<const int32_t*>(page + kPageHdr);
    float v[kXMax / 32];
    load_col(a, X, Tp, xl, nx, 0, v);
    store_col(nx, v, xb->v[0]);
    for (int c = 0; c < RB && p0 + c < a.R; ++c) {
        const bool more = c + 1 < RB && p0 + c + 1 < a.R;
        if (more) load_col(a, X, Tp, xl, nx, c + 1, v);
        __syncwarp();
        f(xb->v[c & 1], c);
        if (more) store_col(nx, v, xb->v[(c + 1) & 1]);
    }
    __syncwarp();
}

// Phase 1: warp w of the grid streams pages [warp_ptr[w], warp_ptr[w + 1]),
// balanced at build time.
template <class T, int RB>
__global__ void __launch_bounds__(256) k_phase1(ApplyArgs a, PageArgs pg, const int32_t* __restrict__ warp_ptr,
                                                const float* const* xsel,
                                                const float* xd, float* __restrict__ Tbuf, float* __restrict__ part,
                                                int* __restrict__ status) {
    // dynamic shared memory: pipes[kWarps], (RB > 1) xbufs[kWarps], carry[kWarps][RB * 128]
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpPipe* pipes = reinterpret_cast<WarpPipe*>(smem_raw);
    XBuf* xbufs = reinterpret_cast<XBuf*>(smem_raw + sizeof(WarpPipe) * kWarps);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* carry = reinterpret_cast<float*>(smem_raw + sizeof(WarpPipe) * kWarps +
                                            (RB > 1 ? sizeof(XBuf) * kWarps : 0)) +
                   warp * RB * 128;
    WarpPipe& wp = pipes[warp];
    const int panel = blockIdx.y, p0 = panel * RB;
    const float* X = (xsel ? *xsel : xd) + (int64_t)p0 * a.n;
    const int64_t gw = (int64_t)blockIdx.x * kWarps + warp;
    const int pa = warp_ptr[gw], pb = warp_ptr[gw + 1];
    const uint32_t lim = g_wait_polls;
    if (lane == 0) {
        pipe_init(wp);
        for (int s = 0; s < kStages && pa + s < pb; ++s) issue_page(pg, pa + s, wp, s);
    }
    __syncwarp();
    int n = 0, issued = min(kStages, pb - pa);
    for (int p = pa; p < pb; ++p, ++n) {
        const int s = n % kStages;
        // warp-uniform decision: a lane that gave up makes the whole warp stop
        if (!__all_sync(0xffffffffu, mbar_wait(&wp.bar[s], (uint32_t)((n / kStages) & 1), lim))) {
            drain(wp, n, issued);  // no bulk copy may stay in flight into this warp's stages
            if (lane == 0) atomicCAS(status, 0, (int)VF_E_TIMEOUT);
            return;
        }
        unsigned char* page = wp.buf[s];
        page_columns<RB>(a, X, nullptr, page, xbufs + warp, p0, [&](const float* xv, int c) {
            for_records<T>(page, [&](const unsigned char* rec) {
                p1_column<T, RB>(a, xv, rec, c, Tbuf, part, carry, panel);
            });
        });
        if (RB == 1) fence_proxy_async_smem();  // the gather wrote the stage; the next copy refills it
        __syncwarp();
        if (p + kStages < pb) {
            if (lane == 0) issue_page(pg, p + kStages, wp, s);
            ++issued;
        }
    }
}

// ------------------------------------------------------------ phase 2
enum { MODE_APPLY = 0, MODE_JACOBI = 1, MODE_RESID = 2 };

struct SweepIO {
    const float* const* xsel;  // indirect: the current input (B_k), tree order (or NULL)
    float* const* ysel;        // indirect: the output buffer (or NULL)
    const float* xd;           // direct input when xsel is NULL
    float* yd;                 // direct output when ysel is NULL
    const float* E;            // tree order, n x R
    const float* rho;          // tree order, n
    double* colpart;           // per (tile, column): sum of squares
    int64_t ntiles;
    int* status;               // VF_E_TIMEOUT if a wait gave up
};

// A column-major slab (cnt <= 64 rows x w columns, element (r, k) at
// k * cnt + r) times its x values: lane r owns slab row r (and r + 32).
// slot: the warp's row slots of this column, stride S.
template <class T, int S, class acc_t, bool SVD>
__device__ __forceinline__ void slab_compute(const float* xv, const T* __restrict__ sA, int cnt, int w, int xb,
                                             const unsigned char* rows8, float sc, acc_t* slot) {
    const int lane = threadIdx.x & 31;
    float q0 = 0.f, q1 = 0.f;
    const bool h0 = lane < cnt, h1 = lane + 32 < cnt;
    if (cnt <= 32) {
        if (h0)
#pragma unroll 8
            for (int k = 0; k < w; ++k) q0 = fmaf(lds(sA + k * cnt + lane), xv[xb + k], q0);
    } else {
#pragma unroll 4
        for (int k = 0; k < w; ++k) {
            const float x = xv[xb + k];
            q0 = fmaf(lds(sA + k * cnt + lane), x, q0);
            if (h1) q1 = fmaf(lds(sA + k * cnt + lane + 32), x, q1);
        }
        if (h1) slot[(SVD ? rows8[lane + 32] : lane + 32) * S] += (acc_t)(q1 * sc);
    }
    if (h0) slot[(SVD ? rows8[lane] : lane) * S] += (acc_t)(q0 * sc);
}

// One record, one panel column, into the warp's row slots.
template <class T, int S, class acc_t>
__device__ __forceinline__ void rec_compute(const float* xv, const unsigned char* rec, acc_t* slot) {
    const int lane = threadIdx.x & 31;
    const uint4 h = *reinterpret_cast<const uint4*>(rec);
    const int kind = (int)(h.x & 0xffu), cnt = (int)((h.x >> 8) & 0xffu), roff = (int)(h.x >> 16);
    const int w = (int)h.y, xb = (int)h.z;
    const float sc = __uint_as_float(h.w);
    const unsigned char* body = rec + kRecHdr;
    if (kind == REC_DENSE) {
        slab_compute<T, S, acc_t, false>(xv, reinterpret_cast<const T*>(body), cnt, w, xb, nullptr, sc,
                                         slot + roff * S);
    } else if (kind == REC_SVD) {
        slab_compute<T, S, acc_t, true>(xv, reinterpret_cast<const T*>(body + pad4((uint32_t)cnt)), cnt, w, xb, body,
                                        sc, slot);
    } else if (kind == REC_CSR) {
        const int32_t* sPtr = reinterpret_cast<const int32_t*>(body);
        const T* sA = reinterpret_cast<const T*>(sPtr + cnt + 1);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int r = lane + 32 * hh;
            if (r >= cnt) continue;
            const int k0 = sPtr[r], k1 = sPtr[r + 1];
            float q = 0.f;
#pragma unroll 4
            for (int k = k0; k < k1; ++k) q = fmaf(lds(sA + k), xv[xb + k], q);
            slot[(roff + r) * S] += (acc_t)(q * sc);
        }
    } else {
        // a long CSR row shared by the lanes, reduced by a fixed butterfly
        const T* sA = reinterpret_cast<const T*>(body);
        float q = 0.f;
        for (int k = lane; k < w; k += 32) q = fmaf(lds(sA + k), xv[xb + k], q);
        for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
        if (lane == 0) slot[roff * S] += (acc_t)(q * sc);
    }
}

// Dynamic shared memory of the phase kernels.
template <int RB, class acc_t>
__host__ __device__ constexpr size_t phase2_smem() {
    return sizeof(WarpPipe) * kWarps + (RB > 1 ? sizeof(XBuf) * kWarps : 0) +
           sizeof(acc_t) * kWarps * kTileRows * RB + sizeof(double) * kWarps * RB;
}
template <int RB>
__host__ __device__ constexpr size_t phase1_smem() {
    return sizeof(WarpPipe) * kWarps + (RB > 1 ? sizeof(XBuf) * kWarps : 0) + sizeof(float) * kWarps * RB * 128;
}

// One CTA per row tile (heaviest first) and RHS panel.  Warp w streams the
// tile's pages [ptr[w], ptr[w+1]) (balanced at build time) through its
// prefetch pipeline; the warps' row slots are then added in warp order, and
// the epilogue applies the mode.
template <class T, int RB, int MODE>
__global__ void __launch_bounds__(256, RB == 1 ? 3 : 1) k_phase2(ApplyArgs a, PageArgs pg, const float* __restrict__ Tbuf,
                                                SweepIO io) {
    using acc_t = typename std::conditional<MODE == MODE_RESID, double, float>::type;
    // dynamic shared memory: pipes[kWarps], (RB > 1) xbufs[kWarps],
    // slots[kWarps][kTileRows * RB] (acc_t), colsum[kWarps][RB]
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpPipe* pipes = reinterpret_cast<WarpPipe*>(smem_raw);
    XBuf* xbufs = reinterpret_cast<XBuf*>(smem_raw + sizeof(WarpPipe) * kWarps);
    const size_t o_slots = sizeof(WarpPipe) * kWarps + (RB > 1 ? sizeof(XBuf) * kWarps : 0);
    auto slots = reinterpret_cast<acc_t(*)[kTileRows * RB]>(smem_raw + o_slots);
    auto colsum = reinterpret_cast<double(*)[RB]>(smem_raw + o_slots + sizeof(acc_t) * kWarps * kTileRows * RB);
    const int tile = a.tile_order[blockIdx.x];
    const int panel = blockIdx.y;
    const int p0 = panel * RB;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tf = a.tile_first[tile], tc = a.tile_count[tile];
    const float* Xb = io.xsel ? *io.xsel : io.xd;
    const float* X = Xb + (int64_t)p0 * a.n;  // this panel's columns
    const float* Tp = Tbuf + (int64_t)panel * RB * a.nT;
    WarpPipe& wp = pipes[warp];
    acc_t* slot = slots[warp];
    for (int i = lane; i < kTileRows * RB; i += 32) slot[i] = 0;
    const int pa = a.tile_page_ptr[tile * kWarps + warp], pb = a.tile_page_ptr[tile * kWarps + warp + 1];
    const uint32_t lim = g_wait_polls;
    if (lane == 0) {
        pipe_init(wp);
        for (int s = 0; s < kStages && pa + s < pb; ++s) issue_page(pg, pa + s, wp, s);
    }
    __syncwarp();
    bool ok = true;
    int consumed = 0, issued = min(kStages, pb - pa);
    for (int p = pa, n = 0; p < pb; ++p, ++n) {
        const int s = n % kStages;
        if (!__all_sync(0xffffffffu, mbar_wait(&wp.bar[s], (uint32_t)((n / kStages) & 1), lim))) {
            ok = false;  // warp-uniform: a lane that gave up makes the whole warp stop
            break;
        }
        unsigned char* page = wp.buf[s];
        page_columns<RB>(a, X, Tp, page, xbufs + warp, p0, [&](const float* xv, int c) {
            for_records<T>(page, [&](const unsigned char* rec) { rec_compute<T, RB, acc_t>(xv, rec, slot + c); });
        });
        if (RB == 1) fence_proxy_async_smem();  // the gather wrote the stage; the next copy refills it
        __syncwarp();
        consumed = n + 1;
        if (p + kStages < pb) {
            if (lane == 0) issue_page(pg, p + kStages, wp, s);
            ++issued;
        }
    }
    if (!ok) {
        drain(wp, consumed, issued);  // no bulk copy may stay in flight into this warp's stages
        if (lane == 0) atomicCAS(io.status, 0, (int)VF_E_TIMEOUT);
    }
    __syncthreads();
    double mysum[RB];
#pragma unroll
    for (int c = 0; c < RB; ++c) mysum[c] = 0.0;
    float* Y = io.ysel ? *io.ysel : io.yd;
    for (int e = threadIdx.x; e < tc * RB; e += blockDim.x) {
        const int r = e / RB, c = e - r * RB;
        if (p0 + c >= a.R) continue;
        acc_t y = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) y += slots[w][r * RB + c];
        const int64_t p = tf + r;
        const int64_t o = (int64_t)(p0 + c) * a.n + p;
        if (MODE == MODE_APPLY) {
            Y[o] = (float)y;
        } else if (MODE == MODE_JACOBI) {
            float bn = io.E[o] + io.rho[p] * (float)y;
            float dd = bn - Xb[o];
            Y[o] = bn;
#pragma unroll
            for (int cc = 0; cc < RB; ++cc)
                if (cc == c) mysum[cc] += (double)dd * dd;
        } else {
            double rr = (double)io.E[o] - (double)Xb[o] + (double)io.rho[p] * (double)y;
            Y[o] = (float)rr;
#pragma unroll
            for (int cc = 0; cc < RB; ++cc)
                if (cc == c) mysum[cc] += rr * rr;
        }
    }
    if (MODE != MODE_APPLY) {
#pragma unroll
        for (int c = 0; c < RB; ++c)
            for (int o = 16; o > 0; o >>= 1) mysum[c] += __shfl_xor_sync(0xffffffffu, mysum[c], o);
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < RB; ++c) colsum[warp][c] = mysum[c];
        __syncthreads();
        if (threadIdx.x < RB && p0 + (int)threadIdx.x < a.R) {
            double sm = 0;
            for (int w = 0; w < kWarps; ++w) sm += colsum[w][threadIdx.x];
            io.colpart[(int64_t)(p0 + threadIdx.x) * io.ntiles + tile] = sm;
        }
    }
}

// ------------------------------------------------------------ page packing
// One warp per record: writes its header, its body (from the block pools,
// element type T) and its x-list entries into the page pool.
template <class T>
__global__ void k_pack_pages(const RecSrc* __restrict__ recs, int64_t nrec, const T* __restrict__ val,
                             const int32_t* __restrict__ aux, const float* __restrict__ scales,
                             const int32_t* __restrict__ xtra, unsigned char* __restrict__ pool) {
    const int64_t ri = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (ri >= nrec) return;
    const RecSrc r = recs[ri];
    unsigned char* dst = pool + r.dst;
    int32_t* xl = reinterpret_cast<int32_t*>(pool + r.xdst);
    uint32_t* h = reinterpret_cast<uint32_t*>(dst);
    const float sc = scales ? scales[r.blk] : 1.f;
    if (lane == 0) {
        h[0] = (uint32_t)r.kind | ((uint32_t)r.cnt << 8) | ((uint32_t)r.roff << 16);
        h[1] = (uint32_t)r.w;
        h[2] = (uint32_t)r.xbase;
        h[3] = __float_as_uint(sc);
        if (r.kind == REC_P1) {
            h[4] = (uint32_t)r.chunk;
            h[5] = (uint32_t)r.nchunks;
            h[6] = (uint32_t)r.first;
            h[7] = (uint32_t)r.x;
        }
    }
    if (r.kind == REC_DENSE) {
        T* o = reinterpret_cast<T*>(dst + kRecHdr);
        for (int e = lane; e < r.cnt * r.w; e += 32) o[e] = val[r.val + e];
        for (int k = lane; k < r.w; k += 32) xl[k] = r.x + k;
    } else if (r.kind == REC_SVD && r.csr) {
        // a CSR piece as a dense slab over its nonempty rows and used columns
        // (both sorted, from xtra); the pool was cleared, so absent entries are 0
        const int32_t* rl = xtra + r.idx;
        const int32_t* cl = rl + r.cnt;
        unsigned char* rows = dst + kRecHdr;
        T* o = reinterpret_cast<T*>(dst + kRecHdr + pad4((uint32_t)r.cnt));
        for (int u = lane; u < r.cnt; u += 32) {
            rows[u] = (unsigned char)(rl[u] - r.tile_first);
            const int lr = rl[u] - r.first;  // block-local row
            int k = 0;
            for (int z = aux[r.nz0 + lr]; z < aux[r.nz0 + lr + 1]; ++z) {
                const int col = aux[r.idx2 + z];
                while (k < r.w && cl[k] < col) ++k;  // the row's columns are a sorted subset of cl
                if (k < r.w) o[k * r.cnt + u] = val[r.val + z];
            }
        }
        for (int k = lane; k < r.w; k += 32) xl[k] = cl[k];
    } else if (r.kind == REC_SVD) {
        unsigned char* rows = dst + kRecHdr;
        for (int u = lane; u < r.cnt; u += 32) rows[u] = (unsigned char)(aux[r.idx + u] - r.tile_first);
        // U' rows (row-major in the block pool) become a column-major slab
        T* o = reinterpret_cast<T*>(dst + kRecHdr + pad4((uint32_t)r.cnt));
        for (int e = lane; e < r.cnt * r.w; e += 32) {
            const int u = e / r.w, k = e - u * r.w;
            o[k * r.cnt + u] = val[r.val + e];
        }
        for (int k = lane; k < r.w; k += 32) xl[k] = -1 - (r.x + k);
    } else if (r.kind == REC_CSR) {
        int32_t* ptr = reinterpret_cast<int32_t*>(dst + kRecHdr);
        for (int i = lane; i <= r.cnt; i += 32) ptr[i] = aux[r.idx + i] - r.nz0;
        T* o = reinterpret_cast<T*>(ptr + r.cnt + 1);
        for (int e = lane; e < r.w; e += 32) {
            xl[e] = aux[r.idx2 + r.nz0 + e];
            o[e] = val[r.val + r.nz0 + e];
        }
    } else if (r.kind == REC_CSR_LONG) {
        T* o = reinterpret_cast<T*>(dst + kRecHdr);
        for (int e = lane; e < r.w; e += 32) {
            xl[e] = aux[r.idx2 + r.nz0 + e];
            o[e] = val[r.val + r.nz0 + e];
        }
    } else {  // phase 1
        for (int j = lane; j < r.cnt; j += 32) xl[j] = aux[r.idx2 + j];
        T* o = reinterpret_cast<T*>(dst + kP1Hdr);
        for (int e = lane; e < r.cnt * r.w; e += 32) o[e] = val[r.val + e];
    }
}

__global__ void k_page_headers(const int32_t* __restrict__ nrec, const uint16_t* __restrict__ used,
                               const int32_t* __restrict__ nx, int64_t npages, unsigned char* __restrict__ pool) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= npages) return;
    uint32_t* h = reinterpret_cast<uint32_t*>(pool + p * (int64_t)kPage);
    h[0] = (uint32_t)nrec[p];
    h[1] = used[p];
    h[2] = (uint32_t)nx[p];
    h[3] = 0u;
}

// ------------------------------------------------------------ small kernels
__global__ void k_gather_cols(const float* __restrict__ src, int64_t lds, const int32_t* __restrict__ perm, int64_t n,
                              int R, float* __restrict__ dst) {
    int64_t tot = n * (int64_t)R;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = e / n, t = e - c * n;
        dst[e] = src[c * lds + perm[t]];
    }
}

__global__ void k_scatter_cols(const float* __restrict__ src, const int32_t* __restrict__ perm, int64_t n, int R,
                               float* __restrict__ dst, int64_t ldd, int clamp) {
    int64_t tot = n * (int64_t)R;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = e / n, t = e - c * n;
        float v = src[e];
        if (clamp) v = fmaxf(v, 0.f);
        dst[c * ldd + perm[t]] = v;
    }
}

__global__ void k_gather_rho(const float* __restrict__ rho, float rho_u, const int32_t* __restrict__ perm, int64_t n,
                             float* __restrict__ dst) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) dst[t] = rho ? rho[perm[t]] : rho_u;
}

// Convergence is tracked per "virtual column" v = s R + c: column c of the
// rows of segment s (one mesh of a stacked matrix; a plain matrix is one
// segment), so every mesh and every right-hand side meets its own tolerance.
//
// per virtual column: ||E||^2 over the segment's rows in double, one
// 1024-thread CTA each; thread t sums elements t, t + 1024, ..., then a
// fixed tree (shuffles, then the warps in order), so the result does not
// depend on scheduling
__global__ void __launch_bounds__(1024) k_colnorm2(const float* __restrict__ E, int64_t n, int R,
                                                   const int32_t* __restrict__ seg_row0, double* __restrict__ out) {
    __shared__ double ws[32];
    const int v = blockIdx.x, c = v % R, sg = v / R, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float* e = E + (int64_t)c * n;
    const int64_t r0 = seg_row0[sg], r1 = seg_row0[sg + 1];
    double s = 0;
    // eight independent loads in flight per thread and step (one column is
    // read by one CTA, so latency, not bandwidth, bounds a plain loop)
    for (int64_t t0 = r0; t0 < r1; t0 += 8 * 1024) {
        float x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int64_t t = t0 + k * 1024 + threadIdx.x;
            x[k] = t < r1 ? __ldg(e + t) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) s += (double)x[k] * (double)x[k];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) ws[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0;
        for (int w = 0; w < 32; ++w) sum += ws[w];
        out[v] = sum;
    }
}

struct LoopState {
    int iter;        // sweeps done in this loop
    int max_iter;
    int parity;      // which ping-pong buffer holds B_k
    int unconverged; // columns still above tolerance after the last sweep
    int done_blocks;
    double rtol2;
};

// Column residuals from the tile partials and the loop decision, in one
// CTA (one warp per column, fixed order): the CTA always sets the while
// condition, and `iter < max_iter` bounds the loop.
__global__ void __launch_bounds__(1024) k_sweep_reduce(const double* __restrict__ colpart, int64_t ntiles, int R,
                                                       int nseg, const int32_t* __restrict__ seg_tile0,
                                                       const double* __restrict__ enorm2, double* __restrict__ colres,
                                                       LoopState* st, float* const* bufs, const float** xsel,
                                                       float** ysel, cudaGraphConditionalHandle handle,
                                                       int use_handle) {
    __shared__ int s_unconv;
    if (threadIdx.x == 0) s_unconv = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    int mine = 0;
    for (int v = warp; v < R * nseg; v += nw) {
        const int c = v % R, sg = v / R;
        double s = 0;
        for (int64_t t = seg_tile0[sg] + lane; t < seg_tile0[sg + 1]; t += 32) s += colpart[(int64_t)c * ntiles + t];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            colres[v] = s;
            if (s > st->rtol2 * enorm2[v]) mine++;
        }
    }
    if (lane == 0 && mine) atomicAdd(&s_unconv, mine);
    __syncthreads();
    if (threadIdx.x != 0) return;
    st->iter += 1;
    st->parity ^= 1;
    *xsel = bufs[st->parity];
    *ysel = bufs[st->parity ^ 1];
    st->unconverged = s_unconv;
    bool again = s_unconv > 0 && st->iter < st->max_iter;
    if (use_handle) cudaGraphSetConditional(handle, again ? 1u : 0u);
}

__global__ void k_loop_init(LoopState* st, int max_iter, double rtol2, float* const* bufs, const float** xsel,
                            float** ysel) {
    st->iter = 0;
    st->max_iter = max_iter;
    st->parity = 0;
    st->unconverged = 0;
    st->done_blocks = 0;
    st->rtol2 = rtol2;
    *xsel = bufs[0];
    *ysel = bufs[1];
}

__global__ void k_axpy_inplace(float* __restrict__ y, const float* __restrict__ x, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += x[i];
}

}  // namespace vf

using namespace vf;

// ============================================================ page plan
namespace {

// Pack records (already in their order) into pages of kPage bytes with FP32
// record sizes, which bound the BF16/FP8 sizes; returns the page of each
// record.  A record never straddles pages.
struct PagePlan {
    std::vector<int64_t> page_of;  // per record
    int64_t npages = 0;
};

}  // namespace

static vf_status build_pages(vf_hmat* H, std::vector<vf::RecSrc>& recs, const std::vector<int64_t>& page_of,
                             int64_t npages, bool phase1, const std::vector<int32_t>& xtra) {
    // per element size: offsets inside pages, page headers, pack kernel
    const int es_of[3] = {4, 2, 1};
    for (int prec = 0; prec < 3; ++prec) {
        if (prec == VF_PREC_BF16 && !H->has_bf16) continue;
        if (prec == VF_PREC_FP8 && !H->has_fp8) continue;
        const int es = es_of[prec];
        // page = header | x list (nx entries) | records
        std::vector<int32_t> nrec(npages, 0), nx(npages, 0), xcur(npages, 0);
        for (size_t i = 0; i < recs.size(); ++i) nx[page_of[i]] += (int32_t)vf::rec_xn(recs[i].kind, recs[i].cnt, recs[i].w);
        std::vector<uint16_t> used(npages);
        for (int64_t pg = 0; pg < npages; ++pg) used[pg] = (uint16_t)vf::page_rec0((uint32_t)nx[pg]);
        for (size_t i = 0; i < recs.size(); ++i) {
            const int64_t pg = page_of[i];
            recs[i].xbase = xcur[pg];
            recs[i].xdst = pg * (int64_t)kPage + kPageHdr + 4 * (int64_t)xcur[pg];
            xcur[pg] += (int32_t)vf::rec_xn(recs[i].kind, recs[i].cnt, recs[i].w);
            recs[i].dst = pg * (int64_t)kPage + used[pg];
            const uint32_t u = used[pg] + vf::rec_bytes(recs[i].kind, recs[i].cnt, recs[i].w, es);
            VF_CHECK(u <= (uint32_t)kPage && xcur[pg] <= kXMax, VF_E_INVAL,
                     "page plan overflows a page (%u bytes, %d x entries)", u, xcur[pg]);
            used[pg] = (uint16_t)u;
            nrec[pg]++;
        }
        vf::dbuf<unsigned char>& pool = phase1 ? H->p1pages[prec] : H->pages[prec];
        vf::dbuf<uint16_t>& u = phase1 ? H->p1_used[prec] : H->page_used[prec];
        VF_TRY(pool.alloc(std::max<int64_t>(npages, 1) * kPage));
        VF_TRY_CUDA(cudaMemset(pool.p, 0, std::max<int64_t>(npages, 1) * kPage));
        VF_TRY(u.upload(used));
        if (npages == 0) continue;
        vf::dbuf<int32_t> dn, dx;
        VF_TRY(dn.upload(nrec));
        VF_TRY(dx.upload(nx));
        vf::dbuf<vf::RecSrc> dr;
        VF_TRY(dr.upload(recs));
        vf::dbuf<int32_t> dxt;
        if (!xtra.empty()) VF_TRY(dxt.upload(xtra));
        const int64_t nr = (int64_t)recs.size();
        const unsigned grid = (unsigned)vf::ceil_div(nr * 32, 256);
        if (nr) {
            if (prec == VF_PREC_FP32)
                vf::k_pack_pages<float><<<grid, 256>>>(dr.p, nr, H->val.p, H->aux.p, nullptr, dxt.p, pool.p);
            else if (prec == VF_PREC_BF16)
                vf::k_pack_pages<__nv_bfloat16><<<grid, 256>>>(dr.p, nr, H->val16.p, H->aux.p, nullptr, dxt.p, pool.p);
            else
                vf::k_pack_pages<__nv_fp8_e4m3><<<grid, 256>>>(dr.p, nr, H->val8.p, H->aux.p, H->scale8.p, dxt.p,
                                                                  pool.p);
            VF_TRY_CUDA(cudaGetLastError());
        }
        vf::k_page_headers<<<(unsigned)vf::ceil_div(npages, 256), 256>>>(dn.p, u.p, dx.p, npages, pool.p);
        VF_TRY_CUDA(cudaGetLastError());
        VF_TRY_CUDA(cudaDeviceSynchronize());
    }
    return VF_OK;
}

int64_t vf_hmat::bytes_payload(int prec) const {
    // the stored representation: values (element size es) and index bytes
    const int64_t es = prec == VF_PREC_FP32 ? 4 : prec == VF_PREC_BF16 ? 2 : 1;
    int64_t b = 0;
    for (const vf::HBlock& k : h_blocks) {
        if (k.kind == VF_BLK_DENSE) b += es * k.m * (int64_t)k.n;
        else if (k.kind == VF_BLK_CSR) b += (es + 4) * (int64_t)k.m1 + 4 * ((int64_t)k.m + 1);
        else if (k.kind == VF_BLK_SVD) b += (es * k.q + 4) * ((int64_t)k.m1 + k.n1);
    }
    return b;
}

vf_status vf_hmat::upload_all() {
    // Row tiles are the tree leaves (h_tile_first/count, filled by assembly or
    // load); every block's row range is a union of consecutive tiles.
    std::vector<vf::HBlock>& B = h_blocks;
    const int64_t ntiles = (int64_t)h_tile_first.size();
    if (h_seg_row0.empty()) {
        h_seg_row0 = {0, (int32_t)nf};
        h_seg_tile0 = {0, (int32_t)ntiles};
    }
    VF_TRY(seg_row0.upload(h_seg_row0));
    VF_TRY(seg_tile0.upload(h_seg_tile0));
    std::vector<int32_t> haux;
    if (n_aux > 0) VF_TRY(aux.download(haux));
    std::vector<int32_t> tile_of_row(nf, -1);
    for (int64_t k = 0; k < ntiles; ++k)
        for (int32_t r = h_tile_first[k]; r < h_tile_first[k] + h_tile_count[k]; ++r) tile_of_row[r] = (int32_t)k;
    // ---- phase-2 records per tile (FP32 sizes; each fits a page).  cap leaves
    // room for the 16-byte padding of the page's x list.
    const int64_t cap = kPage - kPageHdr - 16;
    // FP32 bytes of a record in its page: header, body and its x-list entries
    auto tot = [](int kind, int cnt, int w) {
        return (int64_t)vf::rec_bytes(kind, cnt, w, 4) + 4 * (int64_t)vf::rec_xn(kind, cnt, w);
    };
    std::vector<std::vector<vf::RecSrc>> per(ntiles);
    std::vector<int64_t> cost(ntiles, 0);
    std::vector<int32_t> xtra;  // rows and columns of CSR pieces laid out as dense slabs
    std::vector<int32_t> mark;  // per column of the current CSR block: the stamp of the slab that uses it
    int32_t stamp = 1;
    for (const vf::HBlock& b : B)
        if (b.kind == VF_BLK_CSR) mark.resize(std::max<size_t>(mark.size(), (size_t)b.n), 0);
    for (size_t bi = 0; bi < B.size(); ++bi) {
        const vf::HBlock& b = B[bi];
        for (int32_t r = b.r0; r < b.r0 + b.m;) {
            const int32_t k = tile_of_row[r];
            const int32_t tf = h_tile_first[k], tc = h_tile_count[k];
            // the block's rows inside this tile: [rs, re)
            const int32_t rs = std::max(b.r0, tf), re = std::min(b.r0 + b.m, tf + tc);
            const int32_t cnt = re - rs, br = rs - b.r0, troff = rs - tf;
            vf::RecSrc src{};
            src.blk = (int32_t)bi;
            src.tile_first = tf;
            if (b.kind == VF_BLK_DENSE) {
                // the tile's column-major slab, split into column ranges of <= 128
                const int32_t per_cols = (int32_t)std::min<int64_t>(128, (cap - kRecHdr - 15) / (4 * (int64_t)cnt + 4));
                for (int32_t c0 = 0; c0 < b.n; c0 += per_cols) {
                    src.kind = vf::REC_DENSE;
                    src.cnt = cnt;
                    src.roff = troff;
                    src.w = std::min(per_cols, b.n - c0);
                    src.x = b.c0 + c0;
                    src.val = b.off_val + (int64_t)br * b.n + (int64_t)c0 * cnt;
                    per[k].push_back(src);
                }
            } else if (b.kind == VF_BLK_CSR) {
                const int32_t* rp = haux.data() + b.off_aux;
                const int32_t* ci = rp + b.m + 1;
                src.idx2 = (int32_t)(b.off_aux + b.m + 1);
                src.val = b.off_val;
                // The piece as dense slabs over its nonempty rows and the columns
                // they use (greedy in row order, each slab within a page), unless
                // that takes more than 1.6x the bytes of its CSR records.
                std::vector<vf::RecSrc> dense_recs;
                std::vector<int32_t> dense_xtra;
                int64_t dense_bytes = 0;
                bool dense_ok = true;
                {
                    std::vector<int32_t> rows, cols;
                    auto close = [&]() {
                        if (rows.empty()) return;
                        std::sort(cols.begin(), cols.end());
                        vf::RecSrc d = src;
                        d.kind = vf::REC_SVD;
                        d.csr = 1;
                        d.cnt = (int32_t)rows.size();
                        d.w = (int32_t)cols.size();
                        d.idx = (int32_t)(xtra.size() + dense_xtra.size());
                        d.nz0 = (int32_t)b.off_aux;
                        d.first = b.r0;
                        dense_xtra.insert(dense_xtra.end(), rows.begin(), rows.end());
                        dense_xtra.insert(dense_xtra.end(), cols.begin(), cols.end());
                        dense_bytes += tot(vf::REC_SVD, d.cnt, d.w);
                        dense_recs.push_back(d);
                        rows.clear();
                        cols.clear();
                        ++stamp;
                    };
                    for (int32_t i = 0; i < cnt && dense_ok; ++i) {
                        const int32_t lr = br + i;
                        if (rp[lr + 1] == rp[lr]) continue;
                        int32_t fresh = 0;
                        for (int32_t z = rp[lr]; z < rp[lr + 1]; ++z) fresh += mark[ci[z] - b.c0] != stamp;
                        if (!rows.empty() &&
                            tot(vf::REC_SVD, (int)rows.size() + 1, (int)(cols.size() + fresh)) > cap)
                            close();
                        for (int32_t z = rp[lr]; z < rp[lr + 1]; ++z)
                            if (mark[ci[z] - b.c0] != stamp) {
                                mark[ci[z] - b.c0] = stamp;
                                cols.push_back(ci[z]);
                            }
                        rows.push_back(rs + i);
                        if (tot(vf::REC_SVD, (int)rows.size(), (int)cols.size()) > cap) dense_ok = false;
                    }
                    if (dense_ok) close();
                    ++stamp;
                }
                int64_t csr_bytes = 0;
                const size_t first_csr = per[k].size();
                int32_t i = 0;
                while (i < cnt) {
                    const int32_t row = br + i;
                    const int64_t nz_row = rp[row + 1] - rp[row];
                    if (tot(vf::REC_CSR, 1, (int)nz_row) > cap) {
                        // a long row: lanes share it, in pieces that fit a page
                        const int32_t piece = (int32_t)((cap - kRecHdr - 15) / 8);
                        for (int64_t z = rp[row]; z < rp[row + 1]; z += piece) {
                            vf::RecSrc lr = src;
                            lr.kind = vf::REC_CSR_LONG;
                            lr.cnt = 1;
                            lr.roff = troff + i;
                            lr.nz0 = (int32_t)z;
                            lr.w = (int32_t)std::min<int64_t>(piece, rp[row + 1] - z);
                            per[k].push_back(lr);
                        }
                        ++i;
                        continue;
                    }
                    int32_t j = i + 1;
                    while (j < cnt && tot(vf::REC_CSR, j + 1 - i, rp[br + j + 1] - rp[br + i]) <= cap)
                        ++j;
                    vf::RecSrc cr = src;
                    cr.kind = vf::REC_CSR;
                    cr.cnt = j - i;
                    cr.roff = troff + i;
                    cr.idx = (int32_t)(b.off_aux + br + i);
                    cr.nz0 = rp[br + i];
                    cr.w = rp[br + j] - rp[br + i];
                    if (cr.w > 0) per[k].push_back(cr);
                    i = j;
                }
                for (size_t t = first_csr; t < per[k].size(); ++t)
                    csr_bytes += tot(per[k][t].kind, per[k][t].cnt, per[k][t].w);
                // slabs stream more cheaply per byte than CSR rows (no row
                // walks, one gather per column): on the 79k terrain the
                // multiply kept getting faster up to about 1.3-1.6x the CSR bytes
                if (dense_ok && (double)dense_bytes <= 1.6 * (double)csr_bytes) {
                    per[k].resize(first_csr);
                    per[k].insert(per[k].end(), dense_recs.begin(), dense_recs.end());
                    xtra.insert(xtra.end(), dense_xtra.begin(), dense_xtra.end());
                }
            } else {
                const int32_t* rows = haux.data() + b.off_aux;
                int32_t u0 = (int32_t)(std::lower_bound(rows, rows + b.m1, rs) - rows);
                int32_t u1 = (int32_t)(std::lower_bound(rows, rows + b.m1, re) - rows);
                const int32_t per_rows =
                    (int32_t)std::max<int64_t>(1, (cap - kRecHdr - 4 - 15 - 4 * (int64_t)b.q) / (4 * (int64_t)b.q + 1));
                for (int32_t u = u0; u < u1; u += per_rows) {
                    src.kind = vf::REC_SVD;
                    src.cnt = std::min(per_rows, u1 - u);
                    src.w = b.q;
                    src.x = (int32_t)b.off_T;
                    src.val = b.off_val + (int64_t)u * b.q;
                    src.idx = (int32_t)(b.off_aux + u);
                    per[k].push_back(src);
                }
            }
            r = re;
        }
    }
    // each tile's records go to its warps by longest-processing-time first
    // (records by decreasing bytes, each to the least-loaded warp, lowest
    // index on ties); each warp's records are then packed into its own pages
    std::vector<vf::RecSrc> recs;
    std::vector<int64_t> page_of;
    h_tile_page_ptr.assign(ntiles * kWarps + 1, 0);
    int64_t npages = 0;
    for (int64_t k = 0; k < ntiles; ++k) {
        std::vector<int32_t> ord(per[k].size());
        for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int32_t)i;
        auto bytes_of = [&](int32_t i) { return tot(per[k][i].kind, per[k][i].cnt, per[k][i].w); };
        std::stable_sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) { return bytes_of(x) > bytes_of(y); });
        std::vector<std::vector<int32_t>> lists(kWarps);
        int64_t load[kWarps] = {0};
        for (int32_t i : ord) {
            int best = 0;
            for (int w = 1; w < kWarps; ++w)
                if (load[w] < load[best]) best = w;
            lists[best].push_back(i);
            load[best] += bytes_of(i) + vf::kRecCost;
        }
        for (int w = 0; w < kWarps; ++w) {
            h_tile_page_ptr[k * kWarps + w] = (int32_t)npages;
            int64_t fill = cap + 1;  // forces a new page for the first record
            for (int32_t i : lists[w]) {
                const int64_t bsz = bytes_of(i);
                if (fill + bsz > cap) {
                    ++npages;
                    fill = 0;
                }
                recs.push_back(per[k][i]);
                page_of.push_back(npages - 1);
                fill += bsz;
            }
            cost[k] += load[w] > cost[k] ? load[w] - cost[k] : 0;  // the slowest warp bounds the tile
        }
    }
    h_tile_page_ptr[ntiles * kWarps] = (int32_t)npages;
    n_pages = npages;
    VF_TRY(build_pages(this, recs, page_of, npages, false, xtra));
    h_tile_order.resize(ntiles);
    for (int64_t k = 0; k < ntiles; ++k) h_tile_order[k] = (int32_t)k;
    std::stable_sort(h_tile_order.begin(), h_tile_order.end(),
                     [&](int32_t x, int32_t y) { return cost[x] > cost[y]; });
    // ---- phase-1 records: V' rows of each SVD block, <= 128 rows per record
    // (chunk).  A block's chunks form units that one warp runs in order; a
    // block heavier than a quarter of the mean warp load is cut into units of
    // about that size, whose sums meet in k_p1_reduce.
    struct Unit {
        int32_t blk, c0, c1;  // chunks [c0, c1) of block blk
        int64_t cost;
    };
    auto p1_rows = [&](const vf::HBlock& b) {
        return (int32_t)std::min<int64_t>(128, std::max<int64_t>(1, (cap - kP1Hdr - 15) / (4 * (int64_t)b.q + 4)));
    };
    auto chunk_cost = [&](const vf::HBlock& b, int32_t c) {
        const int32_t rows = p1_rows(b);
        const int32_t cnt = std::min(b.n1, (c + 1) * rows) - c * rows;
        return tot(vf::REC_P1, cnt, b.q) + vf::kRecCost;
    };
    int64_t total = 0, nchunks_all = 0;
    for (const vf::HBlock& b : B)
        if (b.kind == VF_BLK_SVD) {
            const int32_t nch = (int32_t)vf::ceil_div(b.n1, p1_rows(b));
            nchunks_all += nch;
            for (int32_t c = 0; c < nch; ++c) total += chunk_cost(b, c);
        }
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || nsm <= 0) nsm = 148;
    n_p1_warps = std::min<int64_t>((int64_t)nsm * 3 * kWarps, vf::ceil_div(nchunks_all, kWarps) * kWarps);
    n_p1_warps = std::max<int64_t>(n_p1_warps, kWarps);
    const int64_t unit_cap = std::max<int64_t>(16384, total / n_p1_warps / 4);
    std::vector<Unit> units;
    std::vector<int32_t> split;  // per cut block: first slot, units, q, T slot, block
    std::vector<int32_t> unit_slot;
    n_part_slots = 0;
    for (size_t bi = 0; bi < B.size(); ++bi) {
        if (B[bi].kind != VF_BLK_SVD) continue;
        const vf::HBlock& b = B[bi];
        const int32_t nch = (int32_t)vf::ceil_div(b.n1, p1_rows(b));
        const size_t u0 = units.size();
        Unit u{(int32_t)bi, 0, 0, 0};
        for (int32_t c = 0; c < nch; ++c) {
            const int64_t cc = chunk_cost(b, c);
            if (u.c1 > u.c0 && u.cost + cc > unit_cap) {
                units.push_back(u);
                u = Unit{(int32_t)bi, c, c, 0};
            }
            u.c1 = c + 1;
            u.cost += cc;
        }
        units.push_back(u);
        const int32_t nu = (int32_t)(units.size() - u0);
        if (nu > 1) {
            split.insert(split.end(), {(int32_t)n_part_slots, nu, b.q, (int32_t)b.off_T, (int32_t)bi});
            for (int32_t k = 0; k < nu; ++k) unit_slot.push_back((int32_t)(n_part_slots + (int64_t)k * b.q));
            n_part_slots += (int64_t)nu * b.q;
        } else {
            unit_slot.push_back(-1);
        }
    }
    // units to warps by longest-processing-time first (heaviest first, each to
    // the least-loaded warp, lowest index on ties); each warp's units then
    // fill its own pages in order
    std::vector<vf::RecSrc> p1;
    std::vector<int64_t> p1_page;
    {
        std::vector<int32_t> ord(units.size());
        for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int32_t)i;
        std::stable_sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) { return units[x].cost > units[y].cost; });
        using Slot = std::pair<int64_t, int32_t>;  // (load, warp): the smallest load, then the lowest warp
        std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
        for (int32_t w = 0; w < (int32_t)n_p1_warps; ++w) heap.push({0, w});
        std::vector<std::vector<int32_t>> lists(n_p1_warps);
        for (int32_t i : ord) {
            Slot sl = heap.top();
            heap.pop();
            lists[sl.second].push_back(i);
            sl.first += units[i].cost;
            heap.push(sl);
        }
        h_p1_warp_ptr.assign(n_p1_warps + 1, 0);
        int64_t np = 0;
        for (int64_t w = 0; w < n_p1_warps; ++w) {
            h_p1_warp_ptr[w] = (int32_t)np;
            int64_t fill = cap + 1;  // forces a new page for the first record
            for (int32_t ui : lists[w]) {
                const Unit& u = units[ui];
                const vf::HBlock& b = B[u.blk];
                const int32_t rows = p1_rows(b);
                for (int32_t c = u.c0; c < u.c1; ++c) {
                    vf::RecSrc rs{};
                    rs.kind = vf::REC_P1;
                    rs.blk = u.blk;
                    rs.w = b.q;
                    rs.cnt = std::min(b.n1, (c + 1) * rows) - c * rows;
                    rs.x = (int32_t)b.off_T;
                    rs.val = b.off_val + (int64_t)b.m1 * b.q + (int64_t)c * rows * b.q;
                    rs.idx2 = (int32_t)(b.off_aux + b.m1 + (int64_t)c * rows);
                    rs.chunk = c - u.c0;
                    rs.nchunks = u.c1 - u.c0;
                    rs.first = unit_slot[ui];
                    const int64_t bsz = tot(rs.kind, rs.cnt, rs.w);
                    if (fill + bsz > cap) {
                        ++np;
                        fill = 0;
                    }
                    p1.push_back(rs);
                    p1_page.push_back(np - 1);
                    fill += bsz;
                }
            }
        }
        h_p1_warp_ptr[n_p1_warps] = (int32_t)np;
        n_p1_pages = np;
    }
    VF_TRY(build_pages(this, p1, p1_page, n_p1_pages, true, {}));
    VF_TRY(p1_warp_ptr.upload(h_p1_warp_ptr));
    n_split = (int64_t)split.size() / 5;
    if (n_split > 0) VF_TRY(p1_split.upload(split));
    VF_TRY(tile_first.upload(h_tile_first));
    VF_TRY(tile_count.upload(h_tile_count));
    VF_TRY(tile_page_ptr.upload(h_tile_page_ptr));
    VF_TRY(tile_order.upload(h_tile_order));
    return VF_OK;
}

namespace vf {

// Workspace for one (R, precision) solve/apply shape, reused across calls.
struct Workspace {
    int R = 0;
    int prec = 0;
    int RB = 0, npanels = 0;
    dbuf<float> Xt, Yt, Et, Bt[2], rho_t, Tbuf, part, Rbuf;
    dbuf<int> status;         // VF_OK, or VF_E_TIMEOUT if a bounded wait gave up
    dbuf<double> colpart, enorm2, colres;
    dbuf<LoopState> loop;
    dbuf<float*> bufs;        // [2] ping-pong pointers
    dbuf<const float*> xsel;  // current input
    dbuf<float*> ysel;        // current output
    // tensor-core path (BF16, R >= kTensorMinR): BF16 panels of 128 RHS, ping-pong, and the T panel
    dbuf<unsigned char> xpan[2], tpan;
    dbuf<unsigned char> xsplit[2], tsplit[2];  // hi / lo panels of the split residual
    dbuf<float> sx8, isx8;                     // FP8 panels: per RHS column scale and its inverse
    dbuf<int> tcount;  // [0]: columns not converged after a tensor sweep; [1]: the reduction's ticket
    int tpanels = 0;
    bool tready = false, sready = false;  // the tensor panels / the split panels are all allocated
    bool cready = false;                  // the CUDA-core multiply's T and partial buffers are allocated
    cudaGraphExec_t graph = nullptr;
    cudaGraphConditionalHandle handle = 0;
    cudaGraphExec_t tgraph = nullptr;  // the tensor-core Jacobi loop
    cudaGraphConditionalHandle thandle = 0;
    cudaEvent_t done = nullptr;
    ~Workspace() {
        if (graph) cudaGraphExecDestroy(graph);
        if (tgraph) cudaGraphExecDestroy(tgraph);
        if (done) cudaEventDestroy(done);
    }
};

struct WsCache {
    std::mutex mu;
    std::map<std::tuple<int, int, int>, std::unique_ptr<Workspace>> m;  // (R, precision, RB)
};

static std::mutex g_cache_mu;
static std::map<const vf_hmat*, std::unique_ptr<WsCache>> g_cache;

static WsCache& cache_for(const vf_hmat* h) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto& p = g_cache[h];
    if (!p) p = std::make_unique<WsCache>();
    return *p;
}

void drop_cache(const vf_hmat* h) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_cache.erase(h);
}

static int pick_rb(int R) {
    if (R <= 1) return 1;
    if (R <= 2) return 2;
    if (R <= 4) return 4;
    return 8;
}

// The autotuner's record for (prec, R), if any.
static bool tuned(const vf_hmat* h, int prec, int R, vf_tune* t) {
    std::lock_guard<std::mutex> lk(h->tune_mu);
    auto it = h->tunes.find({prec, R});
    if (it == h->tunes.end()) return false;
    *t = it->second;
    return true;
}

static int pick_rb_for(const vf_hmat* h, int prec, int R) {
    vf_tune t;
    return tuned(h, prec, R, &t) ? t.rb : pick_rb(R);
}

static ApplyArgs make_args(const vf_hmat* h, int prec, int R) {
    (void)prec;
    ApplyArgs a{};
    a.tile_first = h->tile_first.p;
    a.tile_count = h->tile_count.p;
    a.tile_page_ptr = h->tile_page_ptr.p;
    a.tile_order = h->tile_order.p;
    a.nparts = std::max<int64_t>(h->n_part_slots, 1);
    a.n = h->nf;
    a.nT = std::max<int64_t>(h->n_T, 1);
    a.R = R;
    return a;
}

static vf_status phase2_attrs(int device);

static vf_status ws_get_rb(const vf_hmat* h, int R, int prec, int RB, Workspace** out) {
    WsCache& c = cache_for(h);
    std::lock_guard<std::mutex> lk(c.mu);
    auto key = std::make_tuple(R, prec, RB);
    auto it = c.m.find(key);
    if (it != c.m.end()) {
        *out = it->second.get();
        return VF_OK;
    }
    VF_TRY(phase2_attrs(h->device));
    auto w = std::make_unique<Workspace>();
    w->R = R;
    w->prec = prec;
    w->RB = RB;
    w->npanels = (int)ceil_div(R, w->RB);
    const int64_t n = h->nf, nR = n * (int64_t)R;
    const int64_t ntiles = (int64_t)h->h_tile_first.size();
    VF_TRY(w->Xt.alloc(nR));
    VF_TRY(w->Yt.alloc(nR));
    VF_TRY(w->Et.alloc(nR));
    VF_TRY(w->Bt[0].alloc(nR));
    VF_TRY(w->Bt[1].alloc(nR));
    VF_TRY(w->Rbuf.alloc(nR));
    VF_TRY(w->rho_t.alloc(n));
    VF_TRY(w->colpart.alloc(std::max<int64_t>(ntiles * R, 1)));
    VF_TRY(w->enorm2.alloc((int64_t)R * h->nseg()));
    VF_TRY(w->colres.alloc((int64_t)R * h->nseg()));
    VF_TRY(w->loop.alloc(1));
    VF_TRY(w->status.alloc(1));
    VF_TRY_CUDA(cudaMemset(w->status.p, 0, sizeof(int)));
    VF_TRY(w->bufs.alloc(2));
    VF_TRY(w->xsel.alloc(1));
    VF_TRY(w->ysel.alloc(1));
    float* hb[2] = {w->Bt[0].p, w->Bt[1].p};
    VF_TRY_CUDA(cudaMemcpy(w->bufs.p, hb, sizeof(hb), cudaMemcpyHostToDevice));
    VF_TRY_CUDA(cudaEventCreateWithFlags(&w->done, cudaEventDisableTiming));
    *out = w.get();
    c.m[key] = std::move(w);
    return VF_OK;
}

static vf_status ws_get(const vf_hmat* h, int R, int prec, Workspace** out) {
    return ws_get_rb(h, R, prec, pick_rb_for(h, prec, R), out);
}

template <class T, int RB, int MODE>
static vf_status launch_phase2(dim3 grid, const ApplyArgs& a, PageArgs pg, const float* Tbuf, const SweepIO& io,
                               cudaStream_t st) {
    using acc_t = typename std::conditional<MODE == MODE_RESID, double, float>::type;
    const size_t smem = phase2_smem<RB, acc_t>();
    k_phase2<T, RB, MODE><<<grid, 256, smem, st>>>(a, pg, Tbuf, io);
    return VF_OK;
}

// The dynamic shared-memory opt-in of every phase-2 variant; called once
// per device before any launch or graph capture.
template <class T, int RB, int MODE>
static cudaError_t phase2_attr() {
    using acc_t = typename std::conditional<MODE == MODE_RESID, double, float>::type;
    const size_t smem = phase2_smem<RB, acc_t>();
    return cudaFuncSetAttribute(k_phase2<T, RB, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <class T, int RB>
static cudaError_t phase2_attrs_rb() {
    cudaError_t e = cudaFuncSetAttribute(k_phase1<T, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)phase1_smem<RB>());
    if (e == cudaSuccess) e = phase2_attr<T, RB, MODE_APPLY>();
    if (e == cudaSuccess) e = phase2_attr<T, RB, MODE_JACOBI>();
    if (e == cudaSuccess) e = phase2_attr<T, RB, MODE_RESID>();
    return e;
}

template <class T>
static cudaError_t phase2_attrs_t() {
    cudaError_t e = phase2_attrs_rb<T, 1>();
    if (e == cudaSuccess) e = phase2_attrs_rb<T, 2>();
    if (e == cudaSuccess) e = phase2_attrs_rb<T, 4>();
    if (e == cudaSuccess) e = phase2_attrs_rb<T, 8>();
    return e;
}

static vf_status phase2_attrs(int device) {
    static std::mutex mu;
    static std::vector<int> done;
    std::lock_guard<std::mutex> lk(mu);
    if (std::find(done.begin(), done.end(), device) != done.end()) return VF_OK;
    cudaError_t e = phase2_attrs_t<float>();
    if (e == cudaSuccess) e = phase2_attrs_t<__nv_bfloat16>();
    if (e == cudaSuccess) e = phase2_attrs_t<__nv_fp8_e4m3>();
    VF_CHECK(e == cudaSuccess, VF_E_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    done.push_back(device);
    return VF_OK;
}

// The scratch one multiply uses: T vectors (npanels x RB x nT floats),
// partial sums of cut blocks, the timeout status word and (sweep modes)
// the per-tile residual partials.
struct Scratch {
    int R, RB, npanels;
    float* T;
    float* part;
    int* status;
    double* colpart;
};

template <class T, int RB>
static vf_status launch_multiply_t(const vf_hmat* h, int prec, const ApplyArgs& a, const Scratch* w, int mode,
                                   const float* const* xsel, float* const* ysel, const float* xd, float* yd,
                                   const float* E, const float* rho, cudaStream_t st) {
    const int64_t ntiles = (int64_t)h->h_tile_first.size();
    if (h->n_p1_pages > 0) {
        dim3 g1((unsigned)(h->n_p1_warps / kWarps), (unsigned)w->npanels);
        PageArgs p1{h->p1pages[prec].p, h->p1_used[prec].p};
        k_phase1<T, RB><<<g1, 256, phase1_smem<RB>(), st>>>(a, p1, h->p1_warp_ptr.p, xsel, xd, w->T, w->part,
                                                            w->status);
        if (h->n_split > 0) {
            dim3 gr((unsigned)ceil_div(h->n_split, 8), (unsigned)w->npanels);
            k_p1_reduce<RB><<<gr, 256, 0, st>>>(a, h->p1_split.p, h->n_split,
                                                prec == VF_PREC_FP8 ? h->scale8.p : nullptr, w->part, w->T);
        }
    }
    SweepIO io{xsel, ysel, xd, yd, E, rho, w->colpart, ntiles, w->status};
    dim3 g2((unsigned)ntiles, (unsigned)w->npanels);
    PageArgs pg{h->pages[prec].p, h->page_used[prec].p};
    vf_status s2;
    if (mode == MODE_APPLY) s2 = launch_phase2<T, RB, MODE_APPLY>(g2, a, pg, w->T, io, st);
    else if (mode == MODE_JACOBI) s2 = launch_phase2<T, RB, MODE_JACOBI>(g2, a, pg, w->T, io, st);
    else s2 = launch_phase2<T, RB, MODE_RESID>(g2, a, pg, w->T, io, st);
    VF_TRY(s2);
    VF_TRY_CUDA(cudaGetLastError());
    return VF_OK;
}

template <class T>
static vf_status launch_multiply_rb(const vf_hmat* h, int prec, const ApplyArgs& a, const Scratch* w, int mode,
                                    const float* const* xsel, float* const* ysel, const float* xd, float* yd,
                                    const float* E, const float* rho, cudaStream_t st) {
    switch (w->RB) {
        case 1: return launch_multiply_t<T, 1>(h, prec, a, w, mode, xsel, ysel, xd, yd, E, rho, st);
        case 2: return launch_multiply_t<T, 2>(h, prec, a, w, mode, xsel, ysel, xd, yd, E, rho, st);
        case 4: return launch_multiply_t<T, 4>(h, prec, a, w, mode, xsel, ysel, xd, yd, E, rho, st);
        default: return launch_multiply_t<T, 8>(h, prec, a, w, mode, xsel, ysel, xd, yd, E, rho, st);
    }
}

// One multiply (phase 1 + phase 2) with the given mode, input/output selected
// through device pointers (xsel/ysel) or given directly (xd/yd).
static vf_status launch_multiply_sc(const vf_hmat* h, int prec, const Scratch* w, int mode, const float* const* xsel,
                                    float* const* ysel, const float* xd, float* yd, const float* E, const float* rho,
                                    cudaStream_t st) {
    ApplyArgs a = make_args(h, prec, w->R);
    if (prec == VF_PREC_FP32) return launch_multiply_rb<float>(h, prec, a, w, mode, xsel, ysel, xd, yd, E, rho, st);
    if (prec == VF_PREC_BF16)
        return launch_multiply_rb<__nv_bfloat16>(h, prec, a, w, mode, xsel, ysel, xd, yd, E, rho, st);
    return launch_multiply_rb<__nv_fp8_e4m3>(h, prec, a, w, mode, xsel, ysel, xd, yd, E, rho, st);
}

// The CUDA-core multiply's scratch of a workspace (T vectors of every RHS
// panel, cut-block partials), allocated on its first use: workspaces whose
// multiplies all run on the tensor cores never hold it.
static vf_status ws_scratch(const vf_hmat* h, Workspace* w) {
    if (w->cready) return VF_OK;
    const int64_t nT = std::max<int64_t>(h->n_T, 1);
    VF_TRY(w->Tbuf.alloc((int64_t)w->npanels * w->RB * nT));
    VF_TRY(w->part.alloc((int64_t)w->npanels * w->RB * std::max<int64_t>(h->n_part_slots, 1)));
    w->cready = true;
    return VF_OK;
}

static vf_status launch_multiply(const vf_hmat* h, int prec, Workspace* w, int mode, const float* const* xsel,
                                 float* const* ysel, const float* xd, float* yd, const float* E, const float* rho,
                                 cudaStream_t st) {
    VF_TRY(ws_scratch(h, w));  // a no-op inside graph capture: ensure_graph calls it first
    const Scratch sc{w->R, w->RB, w->npanels, w->Tbuf.p, w->part.p, w->status.p, w->colpart.p};
    return launch_multiply_sc(h, prec, &sc, mode, xsel, ysel, xd, yd, E, rho, st);
}

// Fixed scratch for vf_apply_tree_static: module globals, never allocated at
// call time.
static __device__ __align__(256) float g_static_T[VF_STATIC_T_FLOATS];
static __device__ __align__(256) float g_static_part[VF_STATIC_PART_FLOATS];
static __device__ __align__(256) int g_static_status[4];

struct StaticScratch {
    float* T = nullptr;
    float* part = nullptr;
    int* status = nullptr;
};

// Addresses of the static scratch on a device, resolved once per device.
static vf_status static_scratch(int device, StaticScratch* out) {
    static std::mutex mu;
    static std::map<int, StaticScratch> addrs;
    std::lock_guard<std::mutex> lk(mu);
    auto it = addrs.find(device);
    if (it == addrs.end()) {
        StaticScratch s;
        VF_TRY_CUDA(cudaGetSymbolAddress((void**)&s.T, g_static_T));
        VF_TRY_CUDA(cudaGetSymbolAddress((void**)&s.part, g_static_part));
        VF_TRY_CUDA(cudaGetSymbolAddress((void**)&s.status, g_static_status));
        it = addrs.emplace(device, s).first;
    }
    *out = it->second;
    return VF_OK;
}

// kernels of one multiply: phase 1 (if any SVD block), the chunk reduction
// (if any block was split), phase 2
static int multiply_kernels(const vf_hmat* h) {
    return (h->n_p1_pages > 0 ? 1 : 0) + (h->n_split > 0 ? 1 : 0) + 1;
}

// BF16 multiplies of at least kTensorMinR columns run on the tensor cores,
// unless the autotuner found the CUDA-core path faster for this R.
static bool use_tensor(const vf_hmat* h, int prec, int R) {
    vf_tune t;
    if (tuned(h, prec, R, &t) && !t.tensor) return false;
    return ((prec == VF_PREC_BF16 && h->has_bf16) || (prec == VF_PREC_FP8 && h->has_fp8)) && R >= kTensorMinR;
}

// The tensor page set of a workspace's precision (1: BF16, 3: FP8) and its
// panels' bytes.
static int tset(const Workspace* w) { return w->prec == VF_PREC_FP8 ? 3 : 1; }
static int64_t tpbx(const vf_hmat* h, int S) { return S == 3 ? tensor_panel_bytes_x8(h) : tensor_panel_bytes_x(h); }
static int64_t tpbt(const vf_hmat* h, int S) { return S == 3 ? tensor_panel_bytes_t8(h) : tensor_panel_bytes_t(h); }

// Scales of the FP8 panels of X (columns [0, R), ld, rows through perm):
// headroom 1 for a single multiply, 1/4 for Jacobi iterates (which may grow
// by up to 1 / (1 - rho) over the right-hand side; beyond that the FP8
// values saturate and the refinement's residual corrects them).
static vf_status fp8_scales(const vf_hmat* h, Workspace* w, const float* X, int64_t ld, const int32_t* perm,
                            float headroom, cudaStream_t st) {
    return tensor_fp8_colscale(h, X, ld, perm, w->R, headroom, w->sx8.p, w->isx8.p, st);
}

// The tensor pages (built once per matrix; the handle's lazily built part)
// and this workspace's panels.
static vf_status tensor_ws(const vf_hmat* h, Workspace* w) {
    const int S = tset(w);
    VF_TRY(tensor_prepare(const_cast<vf_hmat*>(h), S));
    if (w->tready) return VF_OK;  // set only once every buffer below exists
    w->tpanels = (int)ceil_div(w->R, kTensorPanel);
    const int64_t bx = tpbx(h, S), bt = tpbt(h, S);
    if (S == 3) {
        VF_TRY(w->sx8.alloc(w->R));
        VF_TRY(w->isx8.alloc(w->R));
    }
    for (int i = 0; i < 2; ++i) {
        VF_TRY(w->xpan[i].alloc((size_t)w->tpanels * bx));
        VF_TRY_CUDA(cudaMemset(w->xpan[i].p, 0, (size_t)w->tpanels * bx));
    }
    // two T panels: multiplies of two RHS panels at once
    VF_TRY(w->tpan.alloc((size_t)2 * bt));
    VF_TRY_CUDA(cudaMemset(w->tpan.p, 0, (size_t)2 * bt));
    VF_TRY(w->tcount.alloc(2));
    VF_TRY_CUDA(cudaMemset(w->tcount.p, 0, 2 * sizeof(int)));
    w->tready = true;
    return VF_OK;
}

// Virtual columns whose last update exceeded rtol ||E||: one CTA per
// virtual column sums the sweep's per-part partials of its segment in a
// fixed order (threads stride the parts, then shuffles, then the warps in
// order) into colres[v], and the last CTA to finish (an acq_rel ticket)
// counts the unconverged ones.
__global__ void __launch_bounds__(256) k_unconverged(const double* __restrict__ colpart, int64_t ntiles, int R,
                                                     int nseg, const int32_t* __restrict__ seg_part0,
                                                     const double* __restrict__ enorm2, double rtol2,
                                                     double* __restrict__ colres, int* __restrict__ count,
                                                     int* __restrict__ ticket) {
    __shared__ double ws[8];
    __shared__ int s_last;
    const int v = blockIdx.x, c = v % R, sg = v / R, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int NV = R * nseg;
    double s = 0;
    for (int64_t t = seg_part0[sg] + threadIdx.x; t < seg_part0[sg + 1]; t += blockDim.x)
        s += colpart[(int64_t)c * ntiles + t];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) ws[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0;
        for (int w = 0; w < 8; ++w) sum += ws[w];
        colres[v] = sum;
        cuda::atomic_ref<int, cuda::thread_scope_device> tk(*ticket);
        s_last = tk.fetch_add(1, cuda::memory_order_acq_rel) == NV - 1;
    }
    __syncthreads();
    if (!s_last) return;
    // the last CTA: every colres is visible (acquired through the ticket)
    int mine = 0;
    for (int vv = threadIdx.x; vv < NV; vv += blockDim.x)
        if (__ldcg(colres + vv) > rtol2 * enorm2[vv]) mine++;
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    __shared__ int wc[8];
    if (lane == 0) wc[warp] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < 8; ++w) tot += wc[w];
        *count = tot;
        *ticket = 0;  // ready for the next sweep
    }
}

// Jacobi on the tensor cores: B_0 = Et, B_{k+1} = Et + rho .* (F_bf16 B_k)
// until every column's update is <= rtol ||Et|| or max_iter sweeps; the
// result is in Bt[*par].  The sweep loop is one CUDA graph per workspace
// (built on first use): a conditional while node whose body is one sweep
// (the multiplies of every RHS panel, each writing B_{k+1} and the next
// BF16 panel from its epilogue) and the column reduction that decides the
// loop.  The ping-pong direction comes from the loop state's parity, which
// the kernels read when they start, so one captured sweep serves both
// directions.  The host synchronises once, after the loop.
static vf_status ensure_tensor_graph(const vf_hmat* h, Workspace* w) {
    if (w->tgraph) return VF_OK;
    const int S = tset(w);
    const int64_t n = h->nf;
    const int64_t ntiles = tensor_parts(h, S);
    const int64_t bx = tpbx(h, S);
    cudaGraph_t g;
    VF_TRY_CUDA(cudaGraphCreate(&g, 0));
    VF_TRY_CUDA(cudaGraphConditionalHandleCreate(&w->thandle, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = w->thandle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    VF_TRY_CUDA(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t cs;
    VF_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    VF_TRY_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    vf_status s = VF_OK;
    const int* par = &w->loop.p->parity;
    for (int p = 0, np; p < w->tpanels && s == VF_OK; p += np) {
        np = p + 1 < w->tpanels ? 2 : 1;  // two RHS panels per multiply where there are two
        TEpi ep{};
        ep.mode = 1;
        ep.n = n;
        ep.R = w->R;
        ep.p0 = p * kTensorPanel;
        ep.E = w->Et.p;
        ep.rho = w->rho_t.p;
        ep.xstride = bx;
        ep.colpart = w->colpart.p;
        ep.ntiles = ntiles;
        // parity 0: B_k in Bt[0] and xpan[0]; parity 1: in Bt[1] and xpan[1]
        ep.Y = w->Bt[1].p;
        ep.Bold = w->Bt[0].p;
        ep.Xnext = w->xpan[1].p + (size_t)p * bx;
        ep.par = par;
        ep.Xalt = w->xpan[1].p + (size_t)p * bx;
        ep.Yalt = w->Bt[0].p;
        ep.Boldalt = w->Bt[1].p;
        ep.Xnextalt = w->xpan[0].p + (size_t)p * bx;
        if (S == 3) {
            ep.sx = w->sx8.p;
            ep.isx = w->isx8.p;
            ep.irs = tensor_fp8_irs(h);
        }
        s = tensor_multiply(h, S, np, w->xpan[0].p + (size_t)p * bx, nullptr, w->tpan.p, nullptr, ep, w->status.p,
                            cs);
    }
    k_sweep_reduce<<<1, 1024, 0, cs>>>(w->colpart.p, ntiles, w->R, h->nseg(), tensor_seg_parts(h, S), w->enorm2.p,
                                       w->colres.p, w->loop.p, w->bufs.p, w->xsel.p, w->ysel.p, w->thandle, 1);
    cudaError_t e1 = cudaGetLastError();
    cudaGraph_t outg;
    cudaError_t e2 = cudaStreamEndCapture(cs, &outg);
    cudaStreamDestroy(cs);
    if (s != VF_OK) { cudaGraphDestroy(g); return s; }
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        cudaGraphDestroy(g);
        set_error("tensor graph capture failed: %s / %s", cudaGetErrorString(e1), cudaGetErrorString(e2));
        return VF_E_CUDA;
    }
    cudaError_t e3 = cudaGraphInstantiate(&w->tgraph, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) {
        set_error("tensor graph instantiate failed: %s", cudaGetErrorString(e3));
        w->tgraph = nullptr;
        return VF_E_CUDA;
    }
    return VF_OK;
}

static vf_status tensor_jacobi_loop(const vf_hmat* h, Workspace* w, int max_iter, double rtol, cudaStream_t st,
                                    int* iters, int* par, int* kernels) {
    VF_TRY(tensor_ws(h, w));
    VF_TRY(ensure_tensor_graph(h, w));
    const int S = tset(w);
    const int64_t n = h->nf, nR = n * (int64_t)w->R;
    const int64_t bx = tpbx(h, S);
    const int NV = w->R * h->nseg();
    VF_TRY_CUDA(cudaMemcpyAsync(w->Bt[0].p, w->Et.p, nR * 4, cudaMemcpyDeviceToDevice, st));
    k_colnorm2<<<(unsigned)NV, 1024, 0, st>>>(w->Et.p, n, w->R, h->seg_row0.p, w->enorm2.p);
    if (S == 3) VF_TRY(fp8_scales(h, w, w->Et.p, n, nullptr, 0.25f, st));
    for (int p = 0; p < w->tpanels; ++p) {
        if (S == 3)
            VF_TRY(tensor_to_panel8(h, w->Et.p, n, nullptr, w->R, p * kTensorPanel, w->sx8.p,
                                    w->xpan[0].p + (size_t)p * bx, st));
        else
            VF_TRY(tensor_to_panel(h, w->Et.p, n, nullptr, w->R, p * kTensorPanel, w->xpan[0].p + (size_t)p * bx,
                                   nullptr, st));
    }
    k_loop_init<<<1, 1, 0, st>>>(w->loop.p, max_iter, rtol * rtol, w->bufs.p, w->xsel.p, w->ysel.p);
    VF_TRY_CUDA(cudaGetLastError());
    *kernels += 2 + w->tpanels + (S == 3 ? 1 : 0);
    if (max_iter > 0) VF_TRY_CUDA(cudaGraphLaunch(w->tgraph, st));
    LoopState ls{};
    VF_TRY_CUDA(cudaMemcpyAsync(&ls, w->loop.p, sizeof(ls), cudaMemcpyDeviceToHost, st));
    VF_TRY_CUDA(cudaStreamSynchronize(st));
    int per_sweep = 1;  // the column reduction
    for (int p = 0, np; p < w->tpanels; p += np) {
        np = p + 1 < w->tpanels ? 2 : 1;
        per_sweep += tensor_kernels(h, S);
    }
    *kernels += ls.iter * per_sweep;
    *iters = ls.iter;
    *par = ls.parity;
    return VF_OK;
}

// The refinement residual on the tensor cores: r = E - B + rho .* (F B) with
// F B formed from the FP32 factors split in two BF16 terms (three products
// per block piece, FP32 accumulation; ~2^-16 relative) and r, its column
// norms in FP64.  B, E: tree order, column-major (ld n); r -> rout;
// per-column ||r||^2 -> w->colres (device).
static vf_status tensor_residual(const vf_hmat* h, Workspace* w, const float* B, const float* E, float* rout,
                                 cudaStream_t st, int* kernels) {
    VF_TRY(tensor_ws(h, w));
    VF_TRY(tensor_prepare(const_cast<vf_hmat*>(h), 2));
    const int64_t n = h->nf, ntiles = tensor_parts(h, 2);
    const int64_t bx = tensor_panel_bytes_x(h), bt = tensor_panel_bytes_t(h);
    if (!w->sready) {  // set only once every split buffer exists
        for (int i = 0; i < 2; ++i) {
            VF_TRY(w->xsplit[i].alloc((size_t)w->tpanels * bx));
            VF_TRY_CUDA(cudaMemset(w->xsplit[i].p, 0, (size_t)w->tpanels * bx));
            VF_TRY(w->tsplit[i].alloc((size_t)2 * bt));  // two T panels: pairs of RHS panels
            VF_TRY_CUDA(cudaMemset(w->tsplit[i].p, 0, (size_t)2 * bt));
        }
        w->sready = true;
    }
    for (int p = 0, np; p < w->tpanels; p += np) {
        np = p + 1 < w->tpanels ? 2 : 1;  // two RHS panels per multiply where there are two
        unsigned char* xh = w->xsplit[0].p + (size_t)p * bx;
        unsigned char* xl = w->xsplit[1].p + (size_t)p * bx;
        for (int q = 0; q < np; ++q)
            VF_TRY(tensor_to_panel(h, B, n, nullptr, w->R, (p + q) * kTensorPanel, xh + (size_t)q * bx,
                                   xl + (size_t)q * bx, st));
        TEpi ep{};
        ep.mode = 2;
        ep.n = n;
        ep.R = w->R;
        ep.p0 = p * kTensorPanel;
        ep.Y = rout;
        ep.E = E;
        ep.rho = w->rho_t.p;
        ep.Bold = B;
        ep.colpart = w->colpart.p;
        ep.ntiles = ntiles;
        VF_TRY(tensor_multiply(h, 2, np, xh, xl, w->tsplit[0].p, w->tsplit[1].p, ep, w->status.p, st));
        *kernels += np + tensor_kernels(h, 2);
    }
    k_unconverged<<<(unsigned)(w->R * h->nseg()), 256, 0, st>>>(w->colpart.p, ntiles, w->R, h->nseg(),
                                                                tensor_seg_parts(h, 2), w->enorm2.p, 0.0, w->colres.p,
                                                                w->tcount.p, w->tcount.p + 1);
    VF_TRY_CUDA(cudaGetLastError());
    *kernels += 1;
    return VF_OK;
}

// Y (tree order, column-major, ld n) = F X on the tensor cores; X column-major
// with ld, rows taken through perm (NULL: already tree order).
static vf_status tensor_apply(const vf_hmat* h, Workspace* w, const float* X, int64_t ld, const int32_t* perm,
                              float* Y, cudaStream_t st) {
    VF_TRY(tensor_ws(h, w));
    const int S = tset(w);
    const int64_t bx = tpbx(h, S);
    if (S == 3) VF_TRY(fp8_scales(h, w, X, ld, perm, 1.f, st));
    for (int p = 0, np; p < w->tpanels; p += np) {
        np = p + 1 < w->tpanels ? 2 : 1;  // two RHS panels per multiply where there are two
        unsigned char* xp = w->xpan[0].p + (size_t)p * bx;
        for (int q = 0; q < np; ++q) {
            if (S == 3)
                VF_TRY(tensor_to_panel8(h, X, ld, perm, w->R, (p + q) * kTensorPanel, w->sx8.p, xp + (size_t)q * bx,
                                        st));
            else
                VF_TRY(tensor_to_panel(h, X, ld, perm, w->R, (p + q) * kTensorPanel, xp + (size_t)q * bx, nullptr,
                                       st));
        }
        TEpi ep{};
        ep.mode = 0;
        ep.n = h->nf;
        ep.R = w->R;
        ep.p0 = p * kTensorPanel;
        ep.Y = Y;
        if (S == 3) {
            ep.sx = w->sx8.p;
            ep.isx = w->isx8.p;
            ep.irs = tensor_fp8_irs(h);
        }
        VF_TRY(tensor_multiply(h, S, np, xp, nullptr, w->tpan.p, nullptr, ep, w->status.p, st));
    }
    return VF_OK;
}

static vf_status check_prec(const vf_hmat* h, int prec) {
    VF_CHECK(prec == VF_PREC_FP32 || (prec == VF_PREC_BF16 && h->has_bf16) || (prec == VF_PREC_FP8 && h->has_fp8),
             VF_E_INVAL, "precision %d was not built for this matrix", prec);
    return VF_OK;
}

// Build (once per workspace) the graph: a while loop whose body is one
// Jacobi sweep plus the column reduction that sets the loop condition.
static vf_status ensure_graph(const vf_hmat* h, Workspace* w) {
    if (w->graph) return VF_OK;
    VF_TRY(ws_scratch(h, w));  // no allocation may happen during the capture below
    cudaGraph_t g;
    VF_TRY_CUDA(cudaGraphCreate(&g, 0));
    VF_TRY_CUDA(cudaGraphConditionalHandleCreate(&w->handle, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = w->handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    VF_TRY_CUDA(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t cs;
    VF_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    VF_TRY_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    vf_status s =
        launch_multiply(h, w->prec, w, MODE_JACOBI, w->xsel.p, w->ysel.p, nullptr, nullptr, w->Et.p, w->rho_t.p, cs);
    const int64_t ntiles = (int64_t)h->h_tile_first.size();
    k_sweep_reduce<<<1, 1024, 0, cs>>>(w->colpart.p, ntiles, w->R, h->nseg(), h->seg_tile0.p, w->enorm2.p,
                                       w->colres.p, w->loop.p, w->bufs.p, w->xsel.p, w->ysel.p, w->handle, 1);
    cudaError_t e1 = cudaGetLastError();
    cudaGraph_t outg;
    cudaError_t e2 = cudaStreamEndCapture(cs, &outg);
    cudaStreamDestroy(cs);
    if (s != VF_OK) { cudaGraphDestroy(g); return s; }
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        cudaGraphDestroy(g);
        set_error("graph capture failed: %s / %s", cudaGetErrorString(e1), cudaGetErrorString(e2));
        return VF_E_CUDA;
    }
    cudaError_t e3 = cudaGraphInstantiate(&w->graph, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) {
        set_error("graph instantiate failed: %s", cudaGetErrorString(e3));
        w->graph = nullptr;
        return VF_E_CUDA;
    }
    return VF_OK;
}

// Jacobi loop on workspace data: Et, rho_t set; on exit Bt[parity] = B.
static vf_status jacobi_loop(const vf_hmat* h, Workspace* w, int max_iter, double rtol, cudaStream_t st,
                             LoopState* hstate, std::vector<double>* colres, std::vector<double>* en2) {
    const int64_t n = h->nf, nR = n * (int64_t)w->R;
    VF_TRY(ensure_graph(h, w));
    // B_0 = E
    const int NV = w->R * h->nseg();
    VF_TRY_CUDA(cudaMemcpyAsync(w->Bt[0].p, w->Et.p, nR * 4, cudaMemcpyDeviceToDevice, st));
    k_colnorm2<<<(unsigned)NV, 1024, 0, st>>>(w->Et.p, n, w->R, h->seg_row0.p, w->enorm2.p);
    k_loop_init<<<1, 1, 0, st>>>(w->loop.p, max_iter, rtol * rtol, w->bufs.p, w->xsel.p, w->ysel.p);
    VF_TRY_CUDA(cudaGetLastError());
    if (max_iter > 0) VF_TRY_CUDA(cudaGraphLaunch(w->graph, st));
    if (hstate) {
        VF_TRY_CUDA(cudaMemcpyAsync(hstate, w->loop.p, sizeof(LoopState), cudaMemcpyDeviceToHost, st));
        if (colres) {
            colres->resize(NV);
            en2->resize(NV);
            VF_TRY_CUDA(cudaMemcpyAsync(colres->data(), w->colres.p, NV * 8, cudaMemcpyDeviceToHost, st));
            VF_TRY_CUDA(cudaMemcpyAsync(en2->data(), w->enorm2.p, NV * 8, cudaMemcpyDeviceToHost, st));
        }
        VF_TRY_CUDA(cudaStreamSynchronize(st));
    }
    return VF_OK;
}

}  // namespace vf

// ============================================================ C ABI
namespace vf {
void drop_stacks_of(const vf_hmat* h);
}

extern "C" void vf_hmat_destroy(vf_hmat* h) {
    if (!h) return;
    device_guard g(h->device);
    vf::drop_stacks_of(h);
    vf::drop_cache(h);
    delete h;
}

extern "C" int64_t vf_hmat_nfacets(const vf_hmat* h) { return h ? h->nf : -1; }

extern "C" vf_status vf_hmat_trim(vf_hmat* h) {
    clear_error();
    VF_CHECK(h, VF_E_INVAL, "vf_hmat_trim: null argument");
    device_guard g(h->device);
    VF_TRY_CUDA(cudaDeviceSynchronize());  // nothing of the handle in flight
    vf::drop_stacks_of(h);
    vf::drop_cache(h);
    vf::tensor_plan_free(h->tplan);
    h->tplan = nullptr;
    return VF_OK;
}

extern "C" vf_status vf_hmat_blocks(const vf_hmat* h, int64_t* nblocks, int32_t* desc) {
    clear_error();
    VF_CHECK(h && nblocks, VF_E_INVAL, "vf_hmat_blocks: null argument");
    *nblocks = (int64_t)h->h_blocks.size();
    if (desc)
        for (size_t i = 0; i < h->h_blocks.size(); ++i) {
            const vf::HBlock& b = h->h_blocks[i];
            int32_t* d = desc + 7 * i;
            d[0] = b.I;
            d[1] = b.J;
            d[2] = b.kind;
            d[3] = b.q;
            d[4] = b.kind == VF_BLK_SVD ? b.m1 : (b.kind == VF_BLK_CSR ? b.m1 : b.m);
            d[5] = b.kind == VF_BLK_SVD ? b.n1 : b.n;
            d[6] = 0;
        }
    return VF_OK;
}

extern "C" int64_t vf_hmat_bytes(const vf_hmat* h, vf_precision p) { return h ? h->bytes_payload(p) : -1; }

extern "C" vf_status vf_apply(const vf_hmat* h, vf_precision prec, const float* X, int64_t ldx, int32_t R, float* Y,
                              int64_t ldy, vf_stream stream) {
    clear_error();
    VF_CHECK(h && X && Y, VF_E_INVAL, "vf_apply: null argument");
    VF_CHECK(R >= 1 && ldx >= h->nf && ldy >= h->nf, VF_E_INVAL, "vf_apply: need R >= 1 and ld >= N");
    VF_TRY(vf::check_prec(h, prec));
    vf_tune tc;
    if (vf::tuned(h, prec, R, &tc) && tc.rhs_block > 0 && tc.rhs_block < R) {
        for (int32_t c0 = 0; c0 < R; c0 += tc.rhs_block)
            VF_TRY(vf_apply(h, prec, X + (int64_t)c0 * ldx, ldx, std::min(tc.rhs_block, R - c0),
                            Y + (int64_t)c0 * ldy, ldy, stream));
        return VF_OK;
    }
    device_guard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    vf::Workspace* w;
    VF_TRY(vf::ws_get(h, R, prec, &w));
    VF_TRY_CUDA(cudaStreamWaitEvent(st, w->done, 0));
    const int64_t n = h->nf;
    if (vf::use_tensor(h, prec, R)) {
        VF_TRY(vf::tensor_apply(h, w, X, ldx, h->perm.p, w->Yt.p, st));
    } else {
        vf::k_gather_cols<<<1024, 256, 0, st>>>(X, ldx, h->perm.p, n, R, w->Xt.p);
        VF_TRY(vf::launch_multiply(h, prec, w, vf::MODE_APPLY, nullptr, nullptr, w->Xt.p, w->Yt.p, nullptr, nullptr, st));
    }
    vf::k_scatter_cols<<<1024, 256, 0, st>>>(w->Yt.p, h->perm.p, n, R, Y, ldy, 0);
    VF_TRY_CUDA(cudaGetLastError());
    VF_TRY_CUDA(cudaEventRecord(w->done, st));
    return VF_OK;
}

extern "C" vf_status vf_apply_tree(const vf_hmat* h, vf_precision prec, const float* Xt, int32_t R, float* Yt,
                                   vf_stream stream) {
    clear_error();
    VF_CHECK(h && Xt && Yt, VF_E_INVAL, "vf_apply_tree: null argument");
    VF_CHECK(R >= 1, VF_E_INVAL, "vf_apply_tree: need R >= 1");
    VF_TRY(vf::check_prec(h, prec));
    vf_tune tc;
    if (vf::tuned(h, prec, R, &tc) && tc.rhs_block > 0 && tc.rhs_block < R) {
        for (int32_t c0 = 0; c0 < R; c0 += tc.rhs_block)
            VF_TRY(vf_apply_tree(h, prec, Xt + (int64_t)c0 * h->nf, std::min(tc.rhs_block, R - c0),
                                 Yt + (int64_t)c0 * h->nf, stream));
        return VF_OK;
    }
    device_guard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    vf::Workspace* w;
    VF_TRY(vf::ws_get(h, R, prec, &w));
    VF_TRY_CUDA(cudaStreamWaitEvent(st, w->done, 0));
    if (vf::use_tensor(h, prec, R))
        VF_TRY(vf::tensor_apply(h, w, Xt, h->nf, nullptr, Yt, st));
    else
        VF_TRY(vf::launch_multiply(h, prec, w, vf::MODE_APPLY, nullptr, nullptr, Xt, Yt, nullptr, nullptr, st));
    VF_TRY_CUDA(cudaEventRecord(w->done, st));
    return VF_OK;
}

extern "C" vf_status vf_apply_tree_static(const vf_hmat* h, vf_precision prec, const float* Xt, int32_t R, float* Yt,
                                          vf_stream stream) {
    clear_error();
    VF_CHECK(h && Xt && Yt, VF_E_INVAL, "vf_apply_tree_static: null argument");
    VF_CHECK(R >= 1, VF_E_INVAL, "vf_apply_tree_static: need R >= 1");
    VF_TRY(vf::check_prec(h, prec));
    const int RB = vf::pick_rb_for(h, prec, R), npanels = (int)vf::ceil_div(R, RB);
    const int64_t nT = std::max<int64_t>(h->n_T, 1);
    const int64_t need_T = (int64_t)npanels * RB * nT;
    const int64_t need_part = (int64_t)npanels * RB * std::max<int64_t>(h->n_part_slots, 1);
    VF_CHECK(need_T <= VF_STATIC_T_FLOATS && need_part <= VF_STATIC_PART_FLOATS, VF_E_INVAL,
             "vf_apply_tree_static: needs %lld T floats (limit %d) and %lld partial floats (limit %d) for R = %d",
             (long long)need_T, VF_STATIC_T_FLOATS, (long long)need_part, VF_STATIC_PART_FLOATS, (int)R);
    device_guard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    vf::StaticScratch ss;
    VF_TRY(vf::static_scratch(h->device, &ss));
    VF_TRY(vf::phase2_attrs(h->device));
    VF_TRY_CUDA(cudaMemsetAsync(ss.status, 0, sizeof(int), st));
    const vf::Scratch sc{R, RB, npanels, ss.T, ss.part, ss.status, nullptr};
    VF_TRY(vf::launch_multiply_sc(h, prec, &sc, vf::MODE_APPLY, nullptr, nullptr, Xt, Yt, nullptr, nullptr, st));
    int hs = 0;
    VF_TRY_CUDA(cudaMemcpyAsync(&hs, ss.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    VF_TRY_CUDA(cudaStreamSynchronize(st));
    VF_CHECK(hs != VF_E_OOB, VF_E_OOB, "vf_apply_tree_static: a device-side bounds check fired");
    VF_CHECK(hs == 0, VF_E_TIMEOUT, "vf_apply_tree_static: a bounded device-side wait gave up");
    return VF_OK;
}

extern "C" vf_status vf_set_wait_limit(int32_t device, int64_t polls) {
    clear_error();
    VF_CHECK(polls <= 0x7fffffffll, VF_E_INVAL, "vf_set_wait_limit: polls must be < 2^31");
    int ndev = 0;
    VF_TRY_CUDA(cudaGetDeviceCount(&ndev));
    VF_CHECK(device >= 0 && device < ndev, VF_E_INVAL, "vf_set_wait_limit: no device %d", (int)device);
    const uint32_t v = polls < 0 ? vf::kWaitLimit : (uint32_t)polls;
    device_guard g(device);
    VF_TRY_CUDA(cudaMemcpyToSymbol(vf::g_wait_polls, &v, sizeof(v)));
    return VF_OK;
}

namespace vf {

static vf_solve_opts solve_defaults(const vf_solve_opts* in) {
    vf_solve_opts o{};
    o.rtol = 1e-6;
    o.max_iter = 100;
    o.precision = VF_PREC_FP32;
    o.refine = 0;
    o.max_refine = 8;
    o.inner_rtol = 1e-3;
    o.clamp = 0;
    o.rho = 0.f;
    if (in) o = *in;
    if (o.max_iter <= 0) o.max_iter = 100;
    if (o.max_refine <= 0) o.max_refine = 8;
    if (!(o.inner_rtol > 0)) o.inner_rtol = 1e-3;
    return o;
}

// What the solve leaves: the result (tree order, column-major, ld nf) and,
// per virtual column (segment, column), its final relative residual.
struct SolveOut {
    float* result = nullptr;
    std::vector<double> rel;
    std::vector<char> conv;
};

// The solve on tree-ordered data (w->Et = E, w->rho_t = rho set): Jacobi
// in the requested precision, or mixed-precision iterative refinement
// around low-precision Jacobi sweeps.  Adds sweeps, refinements and
// kernel counts to S.
static vf_status solve_core(const vf_hmat* h, const vf_solve_opts& o, int R, cudaStream_t st, Workspace* w,
                            vf_solve_stats* S, SolveOut* out) {
    const int64_t n = h->nf, nR = n * (int64_t)R;
    const int nseg = h->nseg(), NV = R * nseg;
    const bool refine = o.refine && o.precision != VF_PREC_FP32;
    const int kps = multiply_kernels(h) + 1;  // one sweep: the multiply and the column reduction
    out->rel.assign(NV, 0.0);
    out->conv.assign(NV, 1);
    auto judge = [&](const std::vector<double>& res2, const std::vector<double>& en2) {
        bool ok = true;
        for (int v = 0; v < NV; ++v) {
            out->rel[v] = en2[v] > 0 ? std::sqrt(res2[v] / en2[v]) : 0.0;
            out->conv[v] = res2[v] <= o.rtol * o.rtol * en2[v];
            ok = ok && out->conv[v];
        }
        return ok;
    };
    if (!refine) {
        LoopState ls{};
        std::vector<double> colres, en2;
        VF_TRY(jacobi_loop(h, w, o.max_iter, o.rtol, st, &ls, &colres, &en2));
        S->sweeps = ls.iter;
        S->kernels += 2 + ls.iter * kps;  // column norms, loop init, the sweeps
        out->result = w->Bt[ls.parity].p;
        judge(colres, en2);
        return VF_OK;
    }
    // Mixed-precision iterative refinement.  Xt keeps E, Yt accumulates B.
    Workspace* w32;
    VF_TRY(ws_get(h, R, VF_PREC_FP32, &w32));
    VF_TRY_CUDA(cudaMemcpyAsync(w->Xt.p, w->Et.p, nR * 4, cudaMemcpyDeviceToDevice, st));  // E (tree order)
    VF_TRY_CUDA(cudaMemsetAsync(w->Yt.p, 0, nR * 4, st));                                 // B = 0
    std::vector<double> en(NV);
    k_colnorm2<<<(unsigned)NV, 1024, 0, st>>>(w->Xt.p, n, R, h->seg_row0.p, w->enorm2.p);
    S->kernels += 1;
    VF_TRY_CUDA(cudaMemcpyAsync(en.data(), w->enorm2.p, NV * 8, cudaMemcpyDeviceToHost, st));
    VF_TRY_CUDA(cudaStreamSynchronize(st));
    // residual workspace shares the FP32 factors; use w32's selection slots
    VF_TRY_CUDA(cudaMemcpyAsync(w32->rho_t.p, w->rho_t.p, n * 4, cudaMemcpyDeviceToDevice, st));
    const bool tensor = use_tensor(h, o.precision, R);
    const int64_t ntiles = (int64_t)h->h_tile_first.size();
    for (int ref = 0; ref <= o.max_refine; ++ref) {
        // r = E - B + rho F B  (FP32 factors, FP64 accumulation); the
        // residual (written to Et) becomes the next inner right-hand side.
        // With B = 0 (the first pass) r = E exactly, already in Et.
        std::vector<double> rr(NV, 0.0);
        if (ref == 0) {
            rr = en;
        } else if (tensor) {
            int kk = 0;
            VF_TRY(tensor_residual(h, w, w->Yt.p, w->Xt.p, w->Et.p, st, &kk));
            S->kernels += kk;
            VF_TRY_CUDA(cudaMemcpyAsync(rr.data(), w->colres.p, NV * 8, cudaMemcpyDeviceToHost, st));
            VF_TRY_CUDA(cudaStreamSynchronize(st));
        } else {
            VF_TRY(launch_multiply(h, VF_PREC_FP32, w32, MODE_RESID, nullptr, nullptr, w->Yt.p, w->Et.p, w->Xt.p,
                                   w32->rho_t.p, st));
            S->kernels += kps - 1;
            std::vector<double> part((size_t)ntiles * R);
            VF_TRY_CUDA(cudaMemcpyAsync(part.data(), w32->colpart.p, part.size() * 8, cudaMemcpyDeviceToHost, st));
            VF_TRY_CUDA(cudaStreamSynchronize(st));
            for (int v = 0; v < NV; ++v) {
                const int c = v % R, sg = v / R;
                for (int32_t tt = h->h_seg_tile0[sg]; tt < h->h_seg_tile0[sg + 1]; ++tt)
                    rr[v] += part[(size_t)c * ntiles + tt];
            }
        }
        const bool ok = judge(rr, en);
        if (ok || ref == o.max_refine) break;
        S->refinements++;
        // delta = (I - rho F_lowprec)^{-1} r, then B += delta
        LoopState l2{};
        if (tensor) {
            int kk = 0;
            VF_TRY(tensor_jacobi_loop(h, w, o.max_iter, o.inner_rtol, st, &l2.iter, &l2.parity, &kk));
            S->kernels += kk + 1;  // the tensor sweeps, then the update
        } else {
            LoopState ls{};
            VF_TRY(jacobi_loop(h, w, o.max_iter, o.inner_rtol, st, &ls, nullptr, nullptr));
            VF_TRY_CUDA(cudaMemcpyAsync(&l2, w->loop.p, sizeof(l2), cudaMemcpyDeviceToHost, st));
            VF_TRY_CUDA(cudaStreamSynchronize(st));
            S->kernels += 2 + l2.iter * kps + 1;  // column norms, loop init, sweeps, the update
        }
        S->sweeps += l2.iter;
        k_axpy_inplace<<<1024, 256, 0, st>>>(w->Yt.p, w->Bt[l2.parity].p, nR);
        VF_TRY_CUDA(cudaGetLastError());
    }
    out->result = w->Yt.p;
    return VF_OK;
}

// A bounded device-side wait that gave up left VF_E_TIMEOUT in a status
// word of the solve's workspaces: read (and clear) them once the stream has
// drained.
static vf_status solve_status(const vf_hmat* h, Workspace* w, int R, bool refine, cudaStream_t st,
                              const char* who) {
    int ws[2] = {0, 0};
    VF_TRY_CUDA(cudaMemcpyAsync(&ws[0], w->status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    Workspace* wr = nullptr;
    if (refine) {
        VF_TRY(ws_get(h, R, VF_PREC_FP32, &wr));
        VF_TRY_CUDA(cudaMemcpyAsync(&ws[1], wr->status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    VF_TRY_CUDA(cudaEventRecord(w->done, st));
    VF_TRY_CUDA(cudaStreamSynchronize(st));
    if (ws[0] || ws[1]) {
        cudaMemsetAsync(w->status.p, 0, sizeof(int), st);
        if (wr) cudaMemsetAsync(wr->status.p, 0, sizeof(int), st);
        cudaStreamSynchronize(st);
        if (ws[0] == VF_E_OOB || ws[1] == VF_E_OOB) {
            set_error("%s: a device-side bounds check fired", who);
            return VF_E_OOB;
        }
        set_error("%s: a bounded device-side wait gave up", who);
        return VF_E_TIMEOUT;
    }
    return VF_OK;
}

// ---- many meshes: one stacked (block-diagonal) matrix, one launch per phase
// Per mesh of a batched solve: where its facet-order E, B and rho live.
struct SegIO {
    const float* E;
    float* B;
    const float* rho;
    int64_t lde, ldb;
    int32_t R, pad;
};

// Et (tree order, N x R over all meshes) from each mesh's E; columns past a
// mesh's own R are zero.  Facet f of mesh s is stacked row seg_row0[s] + f.
__global__ void k_gather_seg(const SegIO* __restrict__ io, const int32_t* __restrict__ seg_row0, int nseg,
                             const int32_t* __restrict__ perm, int64_t n, int R, float* __restrict__ dst) {
    const int64_t tot = n * (int64_t)R;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, t = e - c * n;
        const int32_t f = perm[t];
        int lo = 0, hi = nseg - 1;  // the segment of stacked facet f
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (seg_row0[mid] <= f) lo = mid; else hi = mid - 1;
        }
        const SegIO s = io[lo];
        dst[e] = c < s.R ? s.E[c * s.lde + (f - seg_row0[lo])] : 0.f;
    }
}

__global__ void k_gather_rho_seg(const SegIO* __restrict__ io, const int32_t* __restrict__ seg_row0, int nseg,
                                 float rho_u, const int32_t* __restrict__ perm, int64_t n, float* __restrict__ dst) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int32_t f = perm[t];
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (seg_row0[mid] <= f) lo = mid; else hi = mid - 1;
    }
    dst[t] = io[lo].rho ? io[lo].rho[f - seg_row0[lo]] : rho_u;
}

__global__ void k_scatter_seg(const float* __restrict__ src, const SegIO* __restrict__ io,
                              const int32_t* __restrict__ seg_row0, int nseg, const int32_t* __restrict__ perm,
                              int64_t n, int R, int clamp) {
    const int64_t tot = n * (int64_t)R;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, t = e - c * n;
        const int32_t f = perm[t];
        int lo = 0, hi = nseg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (seg_row0[mid] <= f) lo = mid; else hi = mid - 1;
        }
        const SegIO s = io[lo];
        if (c >= s.R) continue;
        float v = src[e];
        if (clamp) v = fmaxf(v, 0.f);
        s.B[c * s.ldb + (f - seg_row0[lo])] = v;
    }
}

// Stacked matrices built by vf_solve_batched, keyed by the handles' ids
// (dropped when any of them is destroyed).
struct StackEntry {
    std::vector<uint64_t> uids;
    std::unique_ptr<vf_hmat, void (*)(vf_hmat*)> h{nullptr, vf_hmat_destroy};
    dbuf<SegIO> io;
};
// Never destroyed: at process exit the entries are left to the driver, so
// no handle is destroyed (and no cache walked) during static destruction.
static std::mutex& g_stack_mu = *new std::mutex;
static std::vector<std::unique_ptr<StackEntry>>& g_stacks = *new std::vector<std::unique_ptr<StackEntry>>;

void drop_stacks_of(const vf_hmat* h) {
    std::vector<std::unique_ptr<StackEntry>> gone;  // destroyed after the lock is released
    {
        std::lock_guard<std::mutex> lk(g_stack_mu);
        for (auto it = g_stacks.begin(); it != g_stacks.end();) {
            if (std::find((*it)->uids.begin(), (*it)->uids.end(), h->uid) != (*it)->uids.end()) {
                gone.push_back(std::move(*it));
                it = g_stacks.erase(it);
            } else {
                ++it;
            }
        }
    }
}

static vf_status stack_for(const vf_hmat* const* F, int32_t k, StackEntry** out) {
    std::vector<uint64_t> uids(k);
    for (int32_t i = 0; i < k; ++i) uids[i] = F[i]->uid;
    std::lock_guard<std::mutex> lk(g_stack_mu);
    for (auto& e : g_stacks)
        if (e->uids == uids) {
            *out = e.get();
            return VF_OK;
        }
    auto e = std::make_unique<StackEntry>();
    e->uids = uids;
    VF_TRY(e->io.alloc(k));  // before the stack: a failure here destroys no handle under the lock
    vf_hmat* s = nullptr;
    VF_TRY(vf_hmat_stack(F, k, &s));
    e->h.reset(s);
    *out = e.get();
    g_stacks.push_back(std::move(e));
    return VF_OK;
}

}  // namespace vf

extern "C" vf_status vf_solve(const vf_hmat* h, const float* rho, const float* E, int64_t lde, float* B, int64_t ldb,
                              int32_t R, const vf_solve_opts* opts_in, vf_solve_stats* stats, vf_stream stream) {
    clear_error();
    VF_CHECK(h && E && B, VF_E_INVAL, "vf_solve: null argument");
    VF_CHECK(R >= 1 && lde >= h->nf && ldb >= h->nf, VF_E_INVAL, "vf_solve: need R >= 1 and ld >= N");
    const vf_solve_opts o = vf::solve_defaults(opts_in);
    VF_CHECK(o.rtol > 0, VF_E_INVAL, "vf_solve: rtol must be positive");
    VF_TRY(vf::check_prec(h, o.precision));
    vf_tune tc;
    if (vf::tuned(h, o.precision, R, &tc) && tc.rhs_block > 0 && tc.rhs_block < R) {
        // column blocks of the tuned width, one solve each
        vf_solve_stats all{};
        all.converged = 1;
        vf_status worst = VF_OK;
        for (int32_t c0 = 0; c0 < R; c0 += tc.rhs_block) {
            vf_solve_stats sb{};
            const vf_status sc = vf_solve(h, rho, E + (int64_t)c0 * lde, lde, B + (int64_t)c0 * ldb, ldb,
                                          std::min(tc.rhs_block, R - c0), &o, &sb, stream);
            if (sc != VF_OK && sc != VF_E_NOCONV) return sc;
            if (sc == VF_E_NOCONV) worst = sc;
            all.sweeps = std::max(all.sweeps, sb.sweeps);
            all.refinements = std::max(all.refinements, sb.refinements);
            all.kernels += sb.kernels;
            all.max_rel_residual = std::max(all.max_rel_residual, sb.max_rel_residual);
            all.converged = all.converged && sb.converged;
        }
        if (stats) *stats = all;
        if (worst == VF_E_NOCONV)
            vf::set_error("vf_solve: not converged (max rel residual %.3e)", all.max_rel_residual);
        return worst;
    }
    device_guard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = h->nf;
    vf::Workspace* w;
    VF_TRY(vf::ws_get(h, R, o.precision, &w));
    VF_TRY_CUDA(cudaStreamWaitEvent(st, w->done, 0));
    vf::k_gather_cols<<<1024, 256, 0, st>>>(E, lde, h->perm.p, n, R, w->Et.p);
    vf::k_gather_rho<<<(unsigned)vf::ceil_div(n, 256), 256, 0, st>>>(rho, o.rho, h->perm.p, n, w->rho_t.p);
    VF_TRY_CUDA(cudaGetLastError());
    vf_solve_stats S{};
    S.kernels = 3;  // gather E, gather rho, scatter B
    vf::SolveOut so;
    VF_TRY(vf::solve_core(h, o, R, st, w, &S, &so));
    double mx = 0;
    bool ok = true;
    for (size_t v = 0; v < so.rel.size(); ++v) {
        mx = std::max(mx, so.rel[v]);
        ok = ok && so.conv[v];
    }
    S.max_rel_residual = mx;
    S.converged = ok;
    vf::k_scatter_cols<<<1024, 256, 0, st>>>(so.result, h->perm.p, n, R, B, ldb, o.clamp);
    VF_TRY_CUDA(cudaGetLastError());
    VF_TRY(vf::solve_status(h, w, R, o.refine && o.precision != VF_PREC_FP32, st, "vf_solve"));
    if (stats) *stats = S;
    if (!ok) {
        vf::set_error("vf_solve: not converged (max rel residual %.3e)", S.max_rel_residual);
        return VF_E_NOCONV;
    }
    return VF_OK;
}

extern "C" vf_status vf_solve_host(const vf_hmat* h, const float* rho, const float* E, int64_t lde, float* B,
                                   int64_t ldb, int32_t R, const vf_solve_opts* opts, vf_solve_stats* stats,
                                   vf_stream stream) {
    clear_error();
    VF_CHECK(h && E && B, VF_E_INVAL, "vf_solve_host: null argument");
    VF_CHECK(R >= 1 && lde >= h->nf && ldb >= h->nf, VF_E_INVAL, "vf_solve_host: need R >= 1 and ld >= N");
    device_guard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = h->nf;
    float *dE = nullptr, *dB = nullptr, *drho = nullptr;
    vf_status s = VF_OK;
    auto get = [&](float** p, size_t bytes) {
        if (s != VF_OK) return;
        cudaError_t ea = vf::inject_alloc_failure() ? cudaErrorMemoryAllocation : cudaMallocAsync((void**)p, bytes, st);
        if (ea != cudaSuccess) {
            *p = nullptr;
            set_error("vf_solve_host: device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(ea));
            s = ea == cudaErrorMemoryAllocation ? VF_E_NOMEM : VF_E_CUDA;
        }
    };
    get(&dE, n * R * sizeof(float));
    get(&dB, n * R * sizeof(float));
    if (rho) get(&drho, n * sizeof(float));
    cudaError_t e = cudaSuccess;
    if (s == VF_OK) {
        e = cudaMemcpy2DAsync(dE, n * sizeof(float), E, lde * sizeof(float), n * sizeof(float), R,
                              cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && rho) e = cudaMemcpyAsync(drho, rho, n * sizeof(float), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            set_error("vf_solve_host: copy to device failed: %s", cudaGetErrorString(e));
            s = VF_E_CUDA;
        }
    }
    if (s == VF_OK) s = vf_solve(h, drho, dE, n, dB, n, R, opts, stats, stream);
    if (s == VF_OK || s == VF_E_NOCONV) {
        e = cudaMemcpy2DAsync(B, ldb * sizeof(float), dB, n * sizeof(float), n * sizeof(float), R,
                              cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error("vf_solve_host: copy to host failed: %s", cudaGetErrorString(e));
            s = VF_E_CUDA;
        }
    }
    if (dE) cudaFreeAsync(dE, st);
    if (dB) cudaFreeAsync(dB, st);
    if (drho) cudaFreeAsync(drho, st);
    return s;
}

extern "C" vf_status vf_solve_batched(const vf_hmat* const* F, int32_t nmeshes, const float* const* rho,
                                      const float* const* E, const int64_t* lde, float* const* B, const int64_t* ldb,
                                      const int32_t* R, const vf_solve_opts* opts_in, vf_solve_stats* stats,
                                      vf_stream stream) {
    clear_error();
    VF_CHECK(F && E && B && lde && ldb && R && nmeshes >= 1, VF_E_INVAL, "vf_solve_batched: null argument");
    int32_t Rmax = 0;
    for (int32_t k = 0; k < nmeshes; ++k) {
        VF_CHECK(F[k] && E[k] && B[k], VF_E_INVAL, "vf_solve_batched: null argument for mesh %d", (int)k);
        VF_CHECK(F[k]->device == F[0]->device, VF_E_INVAL, "vf_solve_batched: meshes on different devices");
        VF_CHECK(R[k] >= 1 && lde[k] >= F[k]->nf && ldb[k] >= F[k]->nf, VF_E_INVAL,
                 "vf_solve_batched: mesh %d needs R >= 1 and ld >= N", (int)k);
        Rmax = std::max(Rmax, R[k]);
    }
    if (nmeshes == 1) return vf_solve(F[0], rho ? rho[0] : nullptr, E[0], lde[0], B[0], ldb[0], R[0], opts_in, stats,
                                      stream);
    const vf_solve_opts o = vf::solve_defaults(opts_in);
    VF_CHECK(o.rtol > 0, VF_E_INVAL, "vf_solve_batched: rtol must be positive");
    device_guard g(F[0]->device);
    cudaStream_t st = (cudaStream_t)stream;
    vf::StackEntry* se;
    VF_TRY(vf::stack_for(F, nmeshes, &se));
    const vf_hmat* h = se->h.get();
    VF_TRY(vf::check_prec(h, o.precision));
    const int64_t n = h->nf;
    vf::Workspace* w;
    VF_TRY(vf::ws_get(h, Rmax, o.precision, &w));
    VF_TRY_CUDA(cudaStreamWaitEvent(st, w->done, 0));
    std::vector<vf::SegIO> io(nmeshes);
    for (int32_t k = 0; k < nmeshes; ++k)
        io[k] = vf::SegIO{E[k], B[k], rho ? rho[k] : nullptr, lde[k], ldb[k], R[k], 0};
    VF_TRY_CUDA(cudaMemcpyAsync(se->io.p, io.data(), nmeshes * sizeof(vf::SegIO), cudaMemcpyHostToDevice, st));
    vf::k_gather_seg<<<1024, 256, 0, st>>>(se->io.p, h->seg_row0.p, nmeshes, h->perm.p, n, Rmax, w->Et.p);
    vf::k_gather_rho_seg<<<(unsigned)vf::ceil_div(n, 256), 256, 0, st>>>(se->io.p, h->seg_row0.p, nmeshes, o.rho,
                                                                          h->perm.p, n, w->rho_t.p);
    VF_TRY_CUDA(cudaGetLastError());
    vf_solve_stats S{};
    S.kernels = 3;
    vf::SolveOut so;
    VF_TRY(vf::solve_core(h, o, Rmax, st, w, &S, &so));
    vf::k_scatter_seg<<<1024, 256, 0, st>>>(so.result, se->io.p, h->seg_row0.p, nmeshes, h->perm.p, n, Rmax, o.clamp);
    VF_TRY_CUDA(cudaGetLastError());
    VF_TRY(vf::solve_status(h, w, Rmax, o.refine && o.precision != VF_PREC_FP32, st, "vf_solve_batched"));
    bool all = true;
    double worst = 0;
    for (int32_t k = 0; k < nmeshes; ++k) {
        vf_solve_stats sk = S;
        double mx = 0;
        bool ok = true;
        for (int32_t c = 0; c < R[k]; ++c) {
            mx = std::max(mx, so.rel[(size_t)k * Rmax + c]);
            ok = ok && so.conv[(size_t)k * Rmax + c];
        }
        sk.max_rel_residual = mx;
        sk.converged = ok;
        all = all && ok;
        worst = std::max(worst, mx);
        if (stats) stats[k] = sk;
    }
    if (!all) {
        vf::set_error("vf_solve_batched: not converged (max rel residual %.3e)", worst);
        return VF_E_NOCONV;
    }
    return VF_OK;
}

// ============================================================ autotuner
namespace vf {

__global__ void k_fill_uniform(float* __restrict__ x, int64_t n, uint64_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t h = splitmix64(seed ^ ((uint64_t)i * 0x9E3779B97F4A7C15ull));
        x[i] = (float)((double)(h >> 40) * (1.0 / 16777216.0));
    }
}

static vf_status check_tune(const vf_tune& t, int R) {
    VF_CHECK((t.rb == 1 || t.rb == 2 || t.rb == 4 || t.rb == 8) && (t.tensor == 0 || t.tensor == 1) &&
                 t.rhs_block >= 0 && t.rhs_block < R,
             VF_E_INVAL, "vf_tune: rb must be 1, 2, 4 or 8, tensor 0 or 1, rhs_block in [0, R)");
    return VF_OK;
}

static void tune_store(const vf_hmat* h, int prec, int R, const vf_tune& t) {
    std::lock_guard<std::mutex> lk(h->tune_mu);
    h->tunes[{prec, R}] = t;
    if (t.rhs_block > 0) {
        vf_tune b = t;
        b.rhs_block = 0;  // the blocks themselves run whole
        h->tunes[{prec, t.rhs_block}] = b;
    }
}

}  // namespace vf

extern "C" vf_status vf_tune_set(const vf_hmat* h, vf_precision prec, int32_t R, const vf_tune* t) {
    clear_error();
    VF_CHECK(h && t && R >= 1, VF_E_INVAL, "vf_tune_set: null argument or R < 1");
    VF_TRY(vf::check_prec(h, prec));
    VF_TRY(vf::check_tune(*t, R));
    VF_CHECK(!t->tensor || ((prec == VF_PREC_BF16 || prec == VF_PREC_FP8) && R >= vf::kTensorMinR &&
                            (t->rhs_block == 0 || t->rhs_block >= vf::kTensorMinR)),
             VF_E_INVAL, "vf_tune_set: the tensor path needs BF16 or FP8 and >= %d columns", vf::kTensorMinR);
    vf::tune_store(h, prec, R, *t);
    return VF_OK;
}

extern "C" vf_status vf_autotune(const vf_hmat* h, vf_precision prec, int32_t R, vf_tune* out, vf_stream stream) {
    clear_error();
    VF_CHECK(h && R >= 1, VF_E_INVAL, "vf_autotune: null matrix or R < 1");
    VF_TRY(vf::check_prec(h, prec));
    device_guard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = h->nf;
    std::vector<int32_t> widths{R};
    for (int32_t w = 64; w < R; w *= 2) widths.push_back(w);
    vf::dbuf<float> X, Y;
    VF_TRY(X.alloc((size_t)n * R));
    VF_TRY(Y.alloc((size_t)n * R));
    vf::k_fill_uniform<<<1024, 256, 0, st>>>(X.p, n * (int64_t)R, 0x5EEDull);
    VF_TRY_CUDA(cudaGetLastError());
    cudaEvent_t e0, e1;
    VF_TRY_CUDA(cudaEventCreate(&e0));
    VF_TRY_CUDA(cudaEventCreate(&e1));
    vf_tune best{};
    best.us_per_rhs = -1.f;
    vf_status s = VF_OK;
    for (int32_t W : widths) {
        std::vector<vf_tune> cands;
        // RHS tiles up to the width (at 16 columns and more only the widest:
        // a pass then always fills it)
        for (int rb : {1, 2, 4, 8})
            if ((rb == 1 || rb <= W) && (W < 16 || rb == 8)) cands.push_back(vf_tune{rb, 0, W < R ? W : 0, 0.f});
        if (((prec == VF_PREC_BF16 && h->has_bf16) || (prec == VF_PREC_FP8 && h->has_fp8)) && W >= vf::kTensorMinR)
            cands.push_back(vf_tune{vf::pick_rb(W), 1, W < R ? W : 0, 0.f});
        for (vf_tune& c : cands) {
            vf::Workspace* w;
            if ((s = vf::ws_get_rb(h, W, prec, c.rb, &w)) != VF_OK) break;
            auto run = [&]() -> vf_status {
                if (c.tensor) return vf::tensor_apply(h, w, X.p, n, nullptr, Y.p, st);
                return vf::launch_multiply(h, prec, w, vf::MODE_APPLY, nullptr, nullptr, X.p, Y.p, nullptr, nullptr,
                                           st);
            };
            constexpr int kReps = 3;
            if ((s = run()) != VF_OK) break;  // warm-up (and, for the tensor path, its one-time plan)
            cudaEventRecord(e0, st);
            for (int r = 0; r < kReps && s == VF_OK; ++r) s = run();
            cudaEventRecord(e1, st);
            if (s != VF_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                s = VF_E_CUDA;
                vf::set_error("vf_autotune: %s", cudaGetErrorString(cudaGetLastError()));
                break;
            }
            int ws = 0;
            cudaMemcpy(&ws, w->status.p, sizeof(int), cudaMemcpyDeviceToHost);
            if (ws) {
                cudaMemset(w->status.p, 0, sizeof(int));
                s = VF_E_TIMEOUT;
                vf::set_error("vf_autotune: a bounded device-side wait gave up");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            c.us_per_rhs = ms * 1000.f / kReps / (float)W;
            if (best.us_per_rhs < 0.f || c.us_per_rhs < best.us_per_rhs) best = c;
        }
        if (s != VF_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    VF_TRY(s);
    vf::tune_store(h, prec, R, best);
    if (out) *out = best;
    return VF_OK;
}
