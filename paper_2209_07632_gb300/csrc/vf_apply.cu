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
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>

#include "vf_hmat.cuh"

namespace vf {

constexpr int kTileRows = 64;
constexpr int kWarps = 8;
constexpr int kChunkElems = 8192;  // V' values per phase-1 chunk (one warp)

// ------------------------------------------------------------ value loads
template <class T> __device__ __forceinline__ float ld(const T* p);
template <> __device__ __forceinline__ float ld<float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(p));
}
template <> __device__ __forceinline__ float ld<__nv_fp8_e4m3>(const __nv_fp8_e4m3* p) {
    __nv_fp8_e4m3 v;
    v.__x = __ldg(reinterpret_cast<const unsigned char*>(p));
    return float(v);
}

struct ApplyArgs {
    const HBlock* blocks;
    const int32_t* aux;
    const float* scale;        // per-block scale (FP8) or nullptr
    const int32_t* tile_first;
    const int32_t* tile_count;
    const int32_t* tile_item_ptr;
    const TileItem* items;
    const SvdChunk* chunks;
    const int32_t* tile_order;
    int64_t nparts;            // phase-1 partial slots per panel
    int64_t n;                 // facets
    int64_t nT;                // T slots per RHS column
    int R;                     // total RHS columns
};

// Both phases stream their data as flat, contiguous element ranges: the
// lanes of a warp load consecutive values (fully coalesced), multiply by the
// matching x (or T) entries, stage the products in a per-warp scratch of
// 512 / RB elements, then sum whole rows (phase 2) or whole columns (phase 1)
// out of the scratch in a fixed order.  Every sum therefore has one owner
// and one order: results are bit-reproducible with no float atomics.
// per-warp scratch: 512 products for all RHS panel widths
template <int RB> struct Chunk {
    static constexpr int p2 = 512 / RB;                 // phase 2 elements per pass
    static constexpr int p1 = (512 / RB) < 128 ? 128 : 512 / RB;  // phase 1 (holds a whole V' row)
};

// row index of element e in rows of width w: (e + 0.5) / w is at least
// 0.5 / w away from an integer and its FP32 error is below e / w * 2^-23,
// so the truncation is exact for e < 2^22
__device__ __forceinline__ int row_of(int e, float invw) { return (int)(((float)e + 0.5f) * invw); }

// ------------------------------------------------------------ phase 1
// T_b = V'_b^T X[cols_b] for one chunk of V' rows (one warp).  Input X: tree
// order, column-major with leading dimension n, columns [p0, p0 + RB) of
// the panel.  T: per panel RB x nT (column c at c * nT).  A block split into
// several chunks writes chunk partials; the last chunk to finish (atomic
// ticket) adds them in chunk order.
template <class T, int RB>
__device__ __forceinline__ void phase1_warp(const ApplyArgs& a, const T* __restrict__ val, const float* X,
                                            float* __restrict__ Tbuf, float* __restrict__ part,
                                            int* __restrict__ counters, int ci, int panel, float* scr) {
    const int lane = threadIdx.x & 31;
    const SvdChunk ch = a.chunks[ci];
    const HBlock b = a.blocks[ch.blk];
    const int q = b.q;
    const int p0 = panel * RB;
    const T* Vp = val + b.off_val + (int64_t)b.m1 * q;
    const int32_t* cols = a.aux + b.off_aux + b.m1;
    const float sc = a.scale ? a.scale[ch.blk] : 1.f;
    constexpr int kC = Chunk<RB>::p1;
    const int rows_per = kC / q;  // q <= 128 <= kC
    const float invq = 1.f / (float)q;
    float tk[4][RB];
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int c = 0; c < RB; ++c) tk[t][c] = 0.f;
    for (int j0 = ch.j0; j0 < ch.j1; j0 += rows_per) {
        const int nr = min(rows_per, ch.j1 - j0);
        const int L = nr * q;
        const T* src = Vp + (int64_t)j0 * q;
        float v[kC / 32];
        int jl[kC / 32];
#pragma unroll
        for (int i = 0; i < kC / 32; ++i) {
            int e = lane + 32 * i;
            v[i] = e < L ? ld(src + e) : 0.f;
            jl[i] = e < L ? row_of(e, invq) : 0;
        }
#pragma unroll
        for (int i = 0; i < kC / 32; ++i) {
            int e = lane + 32 * i;
            if (e < L) {
                int col = __ldg(cols + j0 + jl[i]);
#pragma unroll
                for (int c = 0; c < RB; ++c) {
                    float x = (p0 + c < a.R) ? __ldg(X + (int64_t)(p0 + c) * a.n + col) : 0.f;
                    scr[c * kC + e] = v[i] * x;
                }
            }
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            int k = lane + 32 * t;
            if (k < q)
                for (int r = 0; r < nr; ++r)
#pragma unroll
                    for (int c = 0; c < RB; ++c) tk[t][c] += scr[c * kC + r * q + k];
        }
        __syncwarp();
    }
    const int64_t panel_T = (int64_t)panel * RB * a.nT;
    if (ch.nchunks == 1) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            int k = lane + 32 * t;
            if (k < q)
#pragma unroll
                for (int c = 0; c < RB; ++c) Tbuf[panel_T + (int64_t)c * a.nT + b.off_T + k] = tk[t][c] * sc;
        }
        return;
    }
    float* mypart = part + ((int64_t)panel * a.nparts + ch.first + ch.chunk) * (RB * 128);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        int k = lane + 32 * t;
        if (k < q)
#pragma unroll
            for (int c = 0; c < RB; ++c) mypart[c * 128 + k] = tk[t][c];
    }
    __threadfence();
    __syncwarp();
    int last = 0;
    if (lane == 0) last = atomicAdd(counters + (int64_t)panel * a.nT + b.off_T, 1) == ch.nchunks - 1;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return;
    __threadfence();
    const float* pb = part + ((int64_t)panel * a.nparts + ch.first) * (RB * 128);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        int k = lane + 32 * t;
        if (k < q)
#pragma unroll
            for (int c = 0; c < RB; ++c) {
                float s = 0.f;
                for (int cc = 0; cc < ch.nchunks; ++cc) s += __ldcg(pb + (int64_t)cc * (RB * 128) + c * 128 + k);
                Tbuf[panel_T + (int64_t)c * a.nT + b.off_T + k] = s * sc;
            }
    }
    if (lane == 0) counters[(int64_t)panel * a.nT + b.off_T] = 0;
}

template <class T, int RB>
__global__ void __launch_bounds__(256, RB <= 2 ? 4 : 2) k_phase1(ApplyArgs a, const T* __restrict__ val,
                                                                const float* const* xsel, const float* xd,
                                                                float* __restrict__ Tbuf, float* __restrict__ part,
                                                                int* __restrict__ counters, int nchunks) {
    __shared__ float scr[kWarps][RB * Chunk<RB>::p1];
    const int warp = threadIdx.x >> 5;
    const int ci = blockIdx.x * kWarps + warp;
    if (ci >= nchunks) return;
    phase1_warp<T, RB>(a, val, xsel ? *xsel : xd, Tbuf, part, counters, ci, blockIdx.y, scr[warp]);
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
};

// One tile item, processed by one warp into the warp's row accumulators.
template <class T, int RB, class acc_t>
__device__ __forceinline__ void item_warp(const ApplyArgs& a, const T* __restrict__ val, const float* X,
                                          const float* Tp, const TileItem& it, int tf, float* scr, acc_t* acc) {
    const int lane = threadIdx.x & 31;
    const float sc = a.scale ? a.scale[it.blk] : 1.f;
    const int p0 = blockIdx.y * RB;
    int L, base = 0;
    const T* src;
    const int32_t* cj = nullptr;
    if (it.kind == VF_BLK_CSR) {
        base = a.aux[it.idx];
        L = a.aux[it.idx + it.cnt] - base;
        src = val + it.val + base;
        cj = a.aux + it.idx2 + base;
    } else {
        L = it.cnt * it.w;
        src = val + it.val;
    }
    const float invw = it.kind == VF_BLK_CSR ? 0.f : 1.f / (float)it.w;
    const bool wide = (int64_t)it.cnt * it.w >= (1 << 22);  // row_of is exact below 2^22 elements
    constexpr int kC = Chunk<RB>::p2;
    for (int cs = 0; cs < L; cs += kC) {
        const int Lc = min(kC, L - cs);
        float v[kC / 32];
        int xi[kC / 32];
#pragma unroll
        for (int i = 0; i < kC / 32; ++i) {
            int e = lane + 32 * i;
            v[i] = e < Lc ? ld(src + cs + e) : 0.f;
        }
#pragma unroll
        for (int i = 0; i < kC / 32; ++i) {
            int e = cs + lane + 32 * i;
            if (it.kind == VF_BLK_CSR) xi[i] = (lane + 32 * i < Lc) ? __ldg(cj + e) : 0;
            else xi[i] = it.xoff + (e - (wide ? e / it.w : row_of(e, invw)) * it.w);
        }
#pragma unroll
        for (int i = 0; i < kC / 32; ++i) {
            int e = lane + 32 * i;
            if (e < Lc) {
#pragma unroll
                for (int c = 0; c < RB; ++c) {
                    float x;
                    if (it.kind == VF_BLK_SVD) x = Tp[(int64_t)c * a.nT + xi[i]];
                    else x = (p0 + c < a.R) ? __ldg(X + (int64_t)(p0 + c) * a.n + xi[i]) : 0.f;
                    scr[c * kC + e] = v[i] * x;
                }
            }
        }
        __syncwarp();
        // whole-row sums out of the scratch: item row j by lane j (and j + 32)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int j = lane + 32 * h;
            if (j < it.cnt) {
                int rs, re;
                if (it.kind == VF_BLK_CSR) {
                    rs = a.aux[it.idx + j] - base;
                    re = a.aux[it.idx + j + 1] - base;
                } else {
                    rs = j * it.w;
                    re = rs + it.w;
                }
                int lo = max(rs, cs) - cs, hi = min(re, cs + Lc) - cs;
                if (lo < hi) {
                    int dest = it.kind == VF_BLK_SVD ? a.aux[it.idx + j] - tf : j;
#pragma unroll
                    for (int c = 0; c < RB; ++c) {
                        float s = 0.f;
                        for (int k = lo; k < hi; ++k) s += scr[c * kC + k];
                        acc[dest * RB + c] += (acc_t)(s * sc);
                    }
                }
            }
        }
        __syncwarp();
    }
}

// One CTA per row tile (heaviest first) and RHS panel.  Warp w takes the
// tile's items w, w + 8, ... in order; the warps' row accumulators are then
// added in warp order, and the epilogue applies the mode.
template <class T, int RB, int MODE>
__global__ void __launch_bounds__(256, RB <= 2 ? 4 : 2) k_phase2(ApplyArgs a, const T* __restrict__ val,
                                                                const float* __restrict__ Tbuf, SweepIO io) {
    using acc_t = typename std::conditional<MODE == MODE_RESID, double, float>::type;
    // dynamic shared memory: acc[kWarps][kTileRows * RB] (acc_t), colsum[kWarps][RB]
    // (double), scr[kWarps][RB * chunk] (float)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto acc = reinterpret_cast<acc_t(*)[kTileRows * RB]>(smem_raw);
    auto colsum = reinterpret_cast<double(*)[RB]>(smem_raw + sizeof(acc_t) * kWarps * kTileRows * RB);
    auto scr = reinterpret_cast<float(*)[RB * Chunk<RB>::p2]>(smem_raw + sizeof(acc_t) * kWarps * kTileRows * RB +
                                                                sizeof(double) * kWarps * RB);
    const int tile = a.tile_order[blockIdx.x];
    const int panel = blockIdx.y;
    const int p0 = panel * RB;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tf = a.tile_first[tile], tc = a.tile_count[tile];
    const float* X = io.xsel ? *io.xsel : io.xd;
    const float* Tp = Tbuf + (int64_t)panel * RB * a.nT;
    for (int i = lane; i < kTileRows * RB; i += 32) acc[warp][i] = 0;
    __syncwarp();
    const int i0 = a.tile_item_ptr[tile], i1 = a.tile_item_ptr[tile + 1];
    int ii = i0 + warp;
    TileItem nxt;
    if (ii < i1) nxt = a.items[ii];
    for (; ii < i1; ii += kWarps) {
        const TileItem it = nxt;
        if (ii + kWarps < i1) nxt = a.items[ii + kWarps];  // prefetch the next descriptor
        item_warp<T, RB, acc_t>(a, val, X, Tp, it, tf, scr[warp], acc[warp]);
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
        for (int w = 0; w < kWarps; ++w) y += acc[w][r * RB + c];
        const int64_t p = tf + r;
        const int64_t o = (int64_t)(p0 + c) * a.n + p;
        if (MODE == MODE_APPLY) {
            Y[o] = (float)y;
        } else if (MODE == MODE_JACOBI) {
            float bn = io.E[o] + io.rho[p] * (float)y;
            float d = bn - X[o];
            Y[o] = bn;
#pragma unroll
            for (int cc = 0; cc < RB; ++cc)
                if (cc == c) mysum[cc] += (double)d * d;
        } else {
            double rr = (double)io.E[o] - (double)X[o] + (double)io.rho[p] * (double)y;
            Y[o] = (float)rr;
#pragma unroll
            for (int cc = 0; cc < RB; ++cc)
                if (cc == c) mysum[cc] += rr * rr;
        }
    }
    if (MODE != MODE_APPLY) {
        // per-column sums: warp butterfly, then warps in order
#pragma unroll
        for (int c = 0; c < RB; ++c)
            for (int o = 16; o > 0; o >>= 1) mysum[c] += __shfl_xor_sync(0xffffffffu, mysum[c], o);
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < RB; ++c) colsum[warp][c] = mysum[c];
        __syncthreads();
        if (threadIdx.x < RB && p0 + (int)threadIdx.x < a.R) {
            double s = 0;
            for (int w = 0; w < kWarps; ++w) s += colsum[w][threadIdx.x];
            io.colpart[(int64_t)(p0 + threadIdx.x) * io.ntiles + tile] = s;
        }
    }
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

// per column: ||E_c||^2 in double, one warp per column
__global__ void k_colnorm2(const float* __restrict__ E, int64_t n, int R, double* __restrict__ out) {
    int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (c >= R) return;
    double s = 0;
    for (int64_t t = lane; t < n; t += 32) {
        double v = E[(int64_t)c * n + t];
        s += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[c] = s;
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
                                                       const double* __restrict__ enorm2, double* __restrict__ colres,
                                                       LoopState* st, float* const* bufs, const float** xsel,
                                                       float** ysel, cudaGraphConditionalHandle handle,
                                                       int use_handle) {
    __shared__ int s_unconv;
    if (threadIdx.x == 0) s_unconv = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    int mine = 0;
    for (int c = warp; c < R; c += nw) {
        double s = 0;
        for (int64_t t = lane; t < ntiles; t += 32) s += colpart[(int64_t)c * ntiles + t];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            colres[c] = s;
            if (s > st->rtol2 * enorm2[c]) mine++;
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

// ============================================================ work lists
vf_status vf_hmat::upload_all() {
    // Row tiles are the tree leaves (h_tile_first/count, filled by assembly or
    // load); every block's row range is a union of consecutive tiles.
    std::vector<vf::HBlock>& B = h_blocks;
    const int64_t ntiles = (int64_t)h_tile_first.size();
    std::vector<int32_t> haux;
    if (n_aux > 0) VF_TRY(aux.download(haux));
    std::vector<int32_t> tile_of_row(nf, -1);
    for (int64_t k = 0; k < ntiles; ++k)
        for (int32_t r = h_tile_first[k]; r < h_tile_first[k] + h_tile_count[k]; ++r) tile_of_row[r] = (int32_t)k;
    std::vector<std::vector<vf::TileItem>> per(ntiles);
    std::vector<int64_t> cost(ntiles, 0);
    for (size_t bi = 0; bi < B.size(); ++bi) {
        const vf::HBlock& b = B[bi];
        for (int32_t r = b.r0; r < b.r0 + b.m;) {
            const int32_t k = tile_of_row[r];
            const int32_t tf = h_tile_first[k], tc = h_tile_count[k], lr0 = tf - b.r0;
            vf::TileItem it{};
            it.kind = b.kind;
            it.blk = (int32_t)bi;
            int64_t work = 0;
            if (b.kind == VF_BLK_DENSE) {
                it.cnt = tc;
                it.w = b.n;
                it.xoff = b.c0;
                it.val = b.off_val + (int64_t)lr0 * b.n;
                work = (int64_t)tc * b.n;
            } else if (b.kind == VF_BLK_CSR) {
                it.cnt = tc;
                it.idx = (int32_t)(b.off_aux + lr0);
                it.idx2 = (int32_t)(b.off_aux + b.m + 1);
                it.val = b.off_val;
                work = haux[b.off_aux + lr0 + tc] - haux[b.off_aux + lr0];
            } else {
                const int32_t* rows = haux.data() + b.off_aux;
                int32_t u0 = (int32_t)(std::lower_bound(rows, rows + b.m1, tf) - rows);
                int32_t u1 = (int32_t)(std::lower_bound(rows, rows + b.m1, tf + tc) - rows);
                it.cnt = u1 - u0;
                it.w = b.q;
                it.xoff = (int32_t)b.off_T;
                it.val = b.off_val + (int64_t)u0 * b.q;
                it.idx = (int32_t)(b.off_aux + u0);
                work = (int64_t)it.cnt * b.q;
            }
            if (it.cnt > 0 && !(b.kind == VF_BLK_CSR && work == 0)) {
                per[k].push_back(it);
                cost[k] += work + 32;
            }
            r = tf + tc;
        }
    }
    h_items.clear();
    h_tile_item_ptr.assign(ntiles + 1, 0);
    for (int64_t k = 0; k < ntiles; ++k) {
        h_tile_item_ptr[k] = (int32_t)h_items.size();
        h_items.insert(h_items.end(), per[k].begin(), per[k].end());
    }
    h_tile_item_ptr[ntiles] = (int32_t)h_items.size();
    h_tile_order.resize(ntiles);
    for (int64_t k = 0; k < ntiles; ++k) h_tile_order[k] = (int32_t)k;
    std::stable_sort(h_tile_order.begin(), h_tile_order.end(),
                     [&](int32_t x, int32_t y) { return cost[x] > cost[y]; });
    // phase-1 chunks of at most kChunkElems V' values, largest first
    h_chunks.clear();
    n_part_slots = 0;
    for (size_t bi = 0; bi < B.size(); ++bi) {
        if (B[bi].kind != VF_BLK_SVD) continue;
        const int32_t rows = std::max<int32_t>(1, kChunkElems / B[bi].q);
        const int32_t nch = (int32_t)vf::ceil_div(B[bi].n1, rows);
        const int32_t first = nch > 1 ? (int32_t)n_part_slots : 0;
        if (nch > 1) n_part_slots += nch;
        for (int32_t c = 0; c < nch; ++c)
            h_chunks.push_back(vf::SvdChunk{(int32_t)bi, c * rows, std::min(B[bi].n1, (c + 1) * rows), c, nch, first});
    }
    std::stable_sort(h_chunks.begin(), h_chunks.end(), [&](const vf::SvdChunk& x, const vf::SvdChunk& y) {
        return (int64_t)(x.j1 - x.j0) * B[x.blk].q > (int64_t)(y.j1 - y.j0) * B[y.blk].q;
    });
    VF_TRY(tile_first.upload(h_tile_first));
    VF_TRY(tile_count.upload(h_tile_count));
    VF_TRY(tile_item_ptr.upload(h_tile_item_ptr));
    VF_TRY(tile_order.upload(h_tile_order));
    VF_TRY(items.upload(h_items));
    VF_TRY(chunks.upload(h_chunks));
    return VF_OK;
}

namespace vf {

// Workspace for one (R, precision) solve/apply shape, reused across calls.
struct Workspace {
    int R = 0;
    int prec = 0;
    int RB = 0, npanels = 0;
    dbuf<float> Xt, Yt, Et, Bt[2], rho_t, Tbuf, part, Rbuf;
    dbuf<int> counters;
    dbuf<double> colpart, enorm2, colres;
    dbuf<LoopState> loop;
    dbuf<float*> bufs;        // [2] ping-pong pointers
    dbuf<const float*> xsel;  // current input
    dbuf<float*> ysel;        // current output
    cudaGraphExec_t graph = nullptr;
    cudaGraphConditionalHandle handle = 0;
    cudaEvent_t done = nullptr;
    ~Workspace() {
        if (graph) cudaGraphExecDestroy(graph);
        if (done) cudaEventDestroy(done);
    }
};

struct WsCache {
    std::mutex mu;
    std::map<std::pair<int, int>, std::unique_ptr<Workspace>> m;
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

static ApplyArgs make_args(const vf_hmat* h, int prec, int R) {
    ApplyArgs a{};
    a.blocks = h->blocks.p;
    a.aux = h->aux.p;
    a.scale = prec == VF_PREC_FP8 ? h->scale8.p : nullptr;
    a.tile_first = h->tile_first.p;
    a.tile_count = h->tile_count.p;
    a.tile_item_ptr = h->tile_item_ptr.p;
    a.items = h->items.p;
    a.chunks = h->chunks.p;
    a.tile_order = h->tile_order.p;
    a.nparts = std::max<int64_t>(h->n_part_slots, 1);
    a.n = h->nf;
    a.nT = std::max<int64_t>(h->n_T, 1);
    a.R = R;
    return a;
}

static vf_status phase2_attrs(int device);

static vf_status ws_get(const vf_hmat* h, int R, int prec, Workspace** out) {
    WsCache& c = cache_for(h);
    std::lock_guard<std::mutex> lk(c.mu);
    auto key = std::make_pair(R, prec);
    auto it = c.m.find(key);
    if (it != c.m.end()) {
        *out = it->second.get();
        return VF_OK;
    }
    VF_TRY(phase2_attrs(h->device));
    auto w = std::make_unique<Workspace>();
    w->R = R;
    w->prec = prec;
    w->RB = pick_rb(R);
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
    int64_t nT = std::max<int64_t>(h->n_T, 1);
    VF_TRY(w->Tbuf.alloc((int64_t)w->npanels * w->RB * nT));
    VF_TRY(w->part.alloc(std::max<int64_t>((int64_t)w->npanels * std::max<int64_t>(h->n_part_slots, 1) * w->RB * 128, 1)));
    VF_TRY(w->counters.alloc((int64_t)w->npanels * nT));
    VF_TRY_CUDA(cudaMemset(w->counters.p, 0, (int64_t)w->npanels * nT * sizeof(int)));
    VF_TRY(w->colpart.alloc(std::max<int64_t>(ntiles * R, 1)));
    VF_TRY(w->enorm2.alloc(R));
    VF_TRY(w->colres.alloc(R));
    VF_TRY(w->loop.alloc(1));
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

template <class T, int RB, int MODE>
static vf_status launch_phase2(dim3 grid, const ApplyArgs& a, const T* val, const float* Tbuf, const SweepIO& io,
                               cudaStream_t st) {
    using acc_t = typename std::conditional<MODE == MODE_RESID, double, float>::type;
    const size_t smem = sizeof(acc_t) * kWarps * kTileRows * RB + sizeof(double) * kWarps * RB +
                        sizeof(float) * kWarps * RB * Chunk<RB>::p2;
    k_phase2<T, RB, MODE><<<grid, 256, smem, st>>>(a, val, Tbuf, io);
    return VF_OK;
}

// The dynamic shared-memory opt-in of every phase-2 variant; called once
// per device before any launch or graph capture.
template <class T, int RB, int MODE>
static cudaError_t phase2_attr() {
    using acc_t = typename std::conditional<MODE == MODE_RESID, double, float>::type;
    const size_t smem = sizeof(acc_t) * kWarps * kTileRows * RB + sizeof(double) * kWarps * RB +
                        sizeof(float) * kWarps * RB * Chunk<RB>::p2;
    return cudaFuncSetAttribute(k_phase2<T, RB, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <class T, int RB>
static cudaError_t phase2_attrs_rb() {
    cudaError_t e = phase2_attr<T, RB, MODE_APPLY>();
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

template <class T, int RB>
static vf_status launch_multiply_t(const vf_hmat* h, const T* val, const ApplyArgs& a, Workspace* w, int mode,
                                   const float* const* xsel, float* const* ysel, const float* xd, float* yd,
                                   const float* E, const float* rho, cudaStream_t st) {
    const int64_t ntiles = (int64_t)h->h_tile_first.size();
    if (!h->h_chunks.empty()) {
        const int nch = (int)h->h_chunks.size();
        dim3 g1((unsigned)ceil_div(nch, kWarps), (unsigned)w->npanels);
        k_phase1<T, RB><<<g1, 256, 0, st>>>(a, val, xsel, xd, w->Tbuf.p, w->part.p, w->counters.p, nch);
    }
    SweepIO io{xsel, ysel, xd, yd, E, rho, w->colpart.p, ntiles};
    dim3 g2((unsigned)ntiles, (unsigned)w->npanels);
    vf_status s2;
    if (mode == MODE_APPLY) s2 = launch_phase2<T, RB, MODE_APPLY>(g2, a, val, w->Tbuf.p, io, st);
    else if (mode == MODE_JACOBI) s2 = launch_phase2<T, RB, MODE_JACOBI>(g2, a, val, w->Tbuf.p, io, st);
    else s2 = launch_phase2<T, RB, MODE_RESID>(g2, a, val, w->Tbuf.p, io, st);
    VF_TRY(s2);
    VF_TRY_CUDA(cudaGetLastError());
    return VF_OK;
}

template <class T>
static vf_status launch_multiply_rb(const vf_hmat* h, const T* val, const ApplyArgs& a, Workspace* w, int mode,
                                    const float* const* xsel, float* const* ysel, const float* xd, float* yd,
                                    const float* E, const float* rho, cudaStream_t st) {
    switch (w->RB) {
        case 1: return launch_multiply_t<T, 1>(h, val, a, w, mode, xsel, ysel, xd, yd, E, rho, st);
        case 2: return launch_multiply_t<T, 2>(h, val, a, w, mode, xsel, ysel, xd, yd, E, rho, st);
        case 4: return launch_multiply_t<T, 4>(h, val, a, w, mode, xsel, ysel, xd, yd, E, rho, st);
        default: return launch_multiply_t<T, 8>(h, val, a, w, mode, xsel, ysel, xd, yd, E, rho, st);
    }
}

// One multiply (phase 1 + phase 2) with the given mode, input/output selected
// through device pointers.
static vf_status launch_multiply(const vf_hmat* h, int prec, Workspace* w, int mode, const float* const* xsel,
                                 float* const* ysel, const float* xd, float* yd, const float* E, const float* rho,
                                 cudaStream_t st) {
    ApplyArgs a = make_args(h, prec, w->R);
    if (prec == VF_PREC_FP32)
        return launch_multiply_rb<float>(h, h->val.p, a, w, mode, xsel, ysel, xd, yd, E, rho, st);
    if (prec == VF_PREC_BF16)
        return launch_multiply_rb<__nv_bfloat16>(h, h->val16.p, a, w, mode, xsel, ysel, xd, yd, E, rho, st);
    return launch_multiply_rb<__nv_fp8_e4m3>(h, h->val8.p, a, w, mode, xsel, ysel, xd, yd, E, rho, st);
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
    k_sweep_reduce<<<1, 1024, 0, cs>>>(
        w->colpart.p, ntiles, w->R, w->enorm2.p, w->colres.p, w->loop.p, w->bufs.p, w->xsel.p, w->ysel.p, w->handle, 1);
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
    VF_TRY_CUDA(cudaMemcpyAsync(w->Bt[0].p, w->Et.p, nR * 4, cudaMemcpyDeviceToDevice, st));
    k_colnorm2<<<(unsigned)ceil_div((int64_t)w->R * 32, 256), 256, 0, st>>>(w->Et.p, n, w->R, w->enorm2.p);
    k_loop_init<<<1, 1, 0, st>>>(w->loop.p, max_iter, rtol * rtol, w->bufs.p, w->xsel.p, w->ysel.p);
    VF_TRY_CUDA(cudaGetLastError());
    if (max_iter > 0) VF_TRY_CUDA(cudaGraphLaunch(w->graph, st));
    if (hstate) {
        VF_TRY_CUDA(cudaMemcpyAsync(hstate, w->loop.p, sizeof(LoopState), cudaMemcpyDeviceToHost, st));
        if (colres) {
            colres->resize(w->R);
            en2->resize(w->R);
            VF_TRY_CUDA(cudaMemcpyAsync(colres->data(), w->colres.p, w->R * 8, cudaMemcpyDeviceToHost, st));
            VF_TRY_CUDA(cudaMemcpyAsync(en2->data(), w->enorm2.p, w->R * 8, cudaMemcpyDeviceToHost, st));
        }
        VF_TRY_CUDA(cudaStreamSynchronize(st));
    }
    return VF_OK;
}

}  // namespace vf

// ============================================================ C ABI
extern "C" void vf_hmat_destroy(vf_hmat* h) {
    if (!h) return;
    device_guard g(h->device);
    vf::drop_cache(h);
    delete h;
}

extern "C" int64_t vf_hmat_nfacets(const vf_hmat* h) { return h ? h->nf : -1; }

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
    device_guard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    vf::Workspace* w;
    VF_TRY(vf::ws_get(h, R, prec, &w));
    VF_TRY_CUDA(cudaStreamWaitEvent(st, w->done, 0));
    const int64_t n = h->nf;
    vf::k_gather_cols<<<1024, 256, 0, st>>>(X, ldx, h->perm.p, n, R, w->Xt.p);
    VF_TRY(vf::launch_multiply(h, prec, w, vf::MODE_APPLY, nullptr, nullptr, w->Xt.p, w->Yt.p, nullptr, nullptr, st));
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
    device_guard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    vf::Workspace* w;
    VF_TRY(vf::ws_get(h, R, prec, &w));
    VF_TRY_CUDA(cudaStreamWaitEvent(st, w->done, 0));
    VF_TRY(vf::launch_multiply(h, prec, w, vf::MODE_APPLY, nullptr, nullptr, Xt, Yt, nullptr, nullptr, st));
    VF_TRY_CUDA(cudaEventRecord(w->done, st));
    return VF_OK;
}

extern "C" vf_status vf_solve(const vf_hmat* h, const float* rho, const float* E, int64_t lde, float* B, int64_t ldb,
                              int32_t R, const vf_solve_opts* opts_in, vf_solve_stats* stats, vf_stream stream) {
    clear_error();
    VF_CHECK(h && E && B, VF_E_INVAL, "vf_solve: null argument");
    VF_CHECK(R >= 1 && lde >= h->nf && ldb >= h->nf, VF_E_INVAL, "vf_solve: need R >= 1 and ld >= N");
    vf_solve_opts o{};
    o.rtol = 1e-6;
    o.max_iter = 100;
    o.precision = VF_PREC_FP32;
    o.refine = 0;
    o.max_refine = 8;
    o.inner_rtol = 1e-3;
    o.clamp = 0;
    o.rho = 0.f;
    if (opts_in) o = *opts_in;
    if (o.max_iter <= 0) o.max_iter = 100;
    if (o.max_refine <= 0) o.max_refine = 8;
    if (!(o.inner_rtol > 0)) o.inner_rtol = 1e-3;
    VF_CHECK(o.rtol > 0, VF_E_INVAL, "vf_solve: rtol must be positive");
    VF_TRY(vf::check_prec(h, o.precision));
    device_guard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = h->nf, nR = n * (int64_t)R;
    vf::Workspace* w;
    VF_TRY(vf::ws_get(h, R, o.precision, &w));
    VF_TRY_CUDA(cudaStreamWaitEvent(st, w->done, 0));
    vf::k_gather_cols<<<1024, 256, 0, st>>>(E, lde, h->perm.p, n, R, w->Et.p);
    vf::k_gather_rho<<<(unsigned)vf::ceil_div(n, 256), 256, 0, st>>>(rho, o.rho, h->perm.p, n, w->rho_t.p);
    VF_TRY_CUDA(cudaGetLastError());
    vf_solve_stats S{};
    vf::LoopState ls{};
    std::vector<double> colres, en2;
    const bool refine = o.refine && o.precision != VF_PREC_FP32;
    float* result = nullptr;
    vf_status status = VF_OK;
    if (!refine) {
        VF_TRY(vf::jacobi_loop(h, w, o.max_iter, o.rtol, st, &ls, &colres, &en2));
        S.sweeps = ls.iter;
        result = w->Bt[ls.parity].p;
        double mx = 0;
        bool ok = true;
        for (int c = 0; c < R; ++c) {
            double rel = en2[c] > 0 ? std::sqrt(colres[c] / en2[c]) : 0.0;
            mx = std::max(mx, rel);
            ok = ok && colres[c] <= o.rtol * o.rtol * en2[c];
        }
        S.max_rel_residual = mx;
        S.converged = ok;
        if (!ok) status = VF_E_NOCONV;
    } else {
        // Mixed-precision iterative refinement.  Xt keeps E, Yt accumulates B.
        vf::Workspace* w32;
        VF_TRY(vf::ws_get(h, R, VF_PREC_FP32, &w32));
        VF_TRY_CUDA(cudaMemcpyAsync(w->Xt.p, w->Et.p, nR * 4, cudaMemcpyDeviceToDevice, st));  // E (tree order)
        VF_TRY_CUDA(cudaMemsetAsync(w->Yt.p, 0, nR * 4, st));                                 // B = 0
        std::vector<double> en(R);
        vf::k_colnorm2<<<(unsigned)vf::ceil_div((int64_t)R * 32, 256), 256, 0, st>>>(w->Xt.p, n, R, w->enorm2.p);
        VF_TRY_CUDA(cudaMemcpyAsync(en.data(), w->enorm2.p, R * 8, cudaMemcpyDeviceToHost, st));
        VF_TRY_CUDA(cudaStreamSynchronize(st));
        // residual workspace shares the FP32 factors; use w32's selection slots
        VF_TRY_CUDA(cudaMemcpyAsync(w32->rho_t.p, w->rho_t.p, n * 4, cudaMemcpyDeviceToDevice, st));
        double mx = 0;
        bool ok = false;
        for (int ref = 0; ref <= o.max_refine; ++ref) {
            // r = E - B + rho F B  (FP32 factors, FP64 accumulation)
            // the residual (written to Et) becomes the next inner right-hand side
            VF_TRY(vf::launch_multiply(h, VF_PREC_FP32, w32, vf::MODE_RESID, nullptr, nullptr, w->Yt.p, w->Et.p,
                                       w->Xt.p, w32->rho_t.p, st));
            const int64_t ntiles = (int64_t)h->h_tile_first.size();
            std::vector<double> part((size_t)ntiles * R), rr(R, 0.0);
            VF_TRY_CUDA(cudaMemcpyAsync(part.data(), w32->colpart.p, part.size() * 8, cudaMemcpyDeviceToHost, st));
            VF_TRY_CUDA(cudaStreamSynchronize(st));
            mx = 0;
            ok = true;
            for (int c = 0; c < R; ++c) {
                for (int64_t tt = 0; tt < ntiles; ++tt) rr[c] += part[(size_t)c * ntiles + tt];
                double rel = en[c] > 0 ? std::sqrt(rr[c] / en[c]) : 0.0;
                mx = std::max(mx, rel);
                ok = ok && rr[c] <= o.rtol * o.rtol * en[c];
            }
            if (ok || ref == o.max_refine) break;
            S.refinements++;
            // delta = (I - rho F_lowprec)^{-1} r, then B += delta
            VF_TRY(vf::jacobi_loop(h, w, o.max_iter, o.inner_rtol, st, &ls, nullptr, nullptr));
            S.sweeps += 0;
            vf::LoopState l2{};
            VF_TRY_CUDA(cudaMemcpyAsync(&l2, w->loop.p, sizeof(l2), cudaMemcpyDeviceToHost, st));
            VF_TRY_CUDA(cudaStreamSynchronize(st));
            S.sweeps += l2.iter;
            vf::k_axpy_inplace<<<1024, 256, 0, st>>>(w->Yt.p, w->Bt[l2.parity].p, nR);
            VF_TRY_CUDA(cudaGetLastError());
        }
        S.max_rel_residual = mx;
        S.converged = ok;
        result = w->Yt.p;
        if (!ok) status = VF_E_NOCONV;
    }
    vf::k_scatter_cols<<<1024, 256, 0, st>>>(result, h->perm.p, n, R, B, ldb, o.clamp);
    VF_TRY_CUDA(cudaGetLastError());
    VF_TRY_CUDA(cudaEventRecord(w->done, st));
    VF_TRY_CUDA(cudaStreamSynchronize(st));
    if (stats) *stats = S;
    if (status == VF_E_NOCONV) vf::set_error("vf_solve: not converged (max rel residual %.3e)", S.max_rel_residual);
    return status;
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
    VF_TRY_CUDA(cudaMallocAsync((void**)&dE, n * R * sizeof(float), st));
    VF_TRY_CUDA(cudaMallocAsync((void**)&dB, n * R * sizeof(float), st));
    if (rho) VF_TRY_CUDA(cudaMallocAsync((void**)&drho, n * sizeof(float), st));
    vf_status s = VF_OK;
    cudaError_t e = cudaMemcpy2DAsync(dE, n * sizeof(float), E, lde * sizeof(float), n * sizeof(float), R,
                                      cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && rho) e = cudaMemcpyAsync(drho, rho, n * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        set_error("vf_solve_host: copy to device failed: %s", cudaGetErrorString(e));
        s = VF_E_CUDA;
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
    cudaFreeAsync(dE, st);
    cudaFreeAsync(dB, st);
    if (drho) cudaFreeAsync(drho, st);
    return s;
}

extern "C" vf_status vf_solve_batched(const vf_hmat* const* F, int32_t nmeshes, const float* const* rho,
                                      const float* const* E, const int64_t* lde, float* const* B, const int64_t* ldb,
                                      const int32_t* R, const vf_solve_opts* opts, vf_solve_stats* stats,
                                      vf_stream stream) {
    clear_error();
    VF_CHECK(F && E && B && lde && ldb && R && nmeshes >= 1, VF_E_INVAL, "vf_solve_batched: null argument");
    vf_status worst = VF_OK;
    for (int32_t k = 0; k < nmeshes; ++k) {
        vf_status s = vf_solve(F[k], rho ? rho[k] : nullptr, E[k], lde[k], B[k], ldb[k], R[k], opts,
                               stats ? stats + k : nullptr, stream);
        if (s != VF_OK && s != VF_E_NOCONV) return s;
        if (s == VF_E_NOCONV) worst = s;
    }
    return worst;
}
