// The multiply on the 5th-generation tensor cores for panels of 128
// right-hand sides (BF16 or FP8 E4M3 factors and right-hand sides, FP32
// accumulation in tensor memory): Algorithm 5 with the block products as
// tcgen05 MMAs.
//
// Formulation (transposed, so the RHS panel is the MMA's M = 128):
//   phase 1, per SVD block:   T^T (128 x q16) = X^T[cols] (128 x K) . V' (K x q16)
//   phase 2, per row tile:    Y^T (128 x 64)  += X^T[cols] (128 x K) . F_IJ^T (K x rows)
//                                            += T^T[q]    (128 x q16) . U'^T (q16 x rows)
// D lives in TMEM (lane = RHS column, column = output row or T slot).  CSR
// blocks are densified; every operand is zero-padded to the MMA's shape.
//
// Operand layout (no swizzle, MN-major, core matrices of 8 K-rows x 16 bytes
// of MN): element (k, mn) at (k / 8) * LBO + (mn / 8) * 128 + (k % 8) * 16 +
// (mn % 8) * 2, with LBO = (MN / 8) * 128 the byte stride between core
// matrices along K and SBO = 128 the stride along MN.  The RHS panels (X and
// T) are kept in global memory in exactly this layout (MN = 128, row groups
// of 8 = 2 KB), so the A operand of any block is one contiguous byte range:
// its column range (or T slots) rounded to 8 rows, fetched by one bulk copy.
// B operands (the matrix) are packed once into "tensor pages" in the same
// layout.  FP8 (kind::f8f6f4) uses K-major operands instead: core matrices
// of 8 MN rows x 16 K bytes, element (mn, k) at (k / 16) * LBO + (mn / 8) *
// 128 + (mn % 8) * 16 + k % 16, LBO = (MN / 8) * 128 along K, SBO = 128 along
// MN, and an MMA step of K = 32; FP8 panels are 128 bytes per row, records
// come in 32-column chunks and every value carries a power-of-two scale
// (per RHS column, per output row, per SVD rank column) that the epilogues
// undo.
//
// Each kernel is persistent (four CTAs per SM, three for the split set)
// with warp roles: warp 0 lane 0 copies pages and A operands
// (cp.async.bulk, mbarrier completion), warp 1 lane 0 issues the MMAs and
// commits them to mbarriers, warps 2-5 read the finished accumulators
// (tcgen05.ld) and run the epilogue.  Two accumulator
// regions alternate between tiles (units), so the epilogue of one overlaps
// the MMAs of the next.  Every wait is bounded; a role that gives up records
// VF_E_TIMEOUT and stops issuing, and the kernel waits (bounded) for work in
// flight before it frees its tensor memory.
#include <algorithm>
#include <cmath>
#include <functional>
#include <memory>
#include <numeric>
#include <queue>
#include <vector>

#include "vf_bulk.cuh"
#include "vf_hmat.cuh"
#include "vf_tensor.cuh"

namespace vf {

#ifndef VF_T_PAGE
#define VF_T_PAGE 12288
#endif
constexpr int kTP = VF_T_PAGE;       // tensor page bytes
constexpr int kTPHdr = 16;           // page header: nrec, used, 0, 0
constexpr int kTRHdr = 32;           // record header (8 x u32)
constexpr int kPanel = 128;          // right-hand sides per panel (MMA M)
constexpr int kMaxSlots = 16;        // A-operand ring slots (barrier pairs)
// Kernel configurations per (NS, NP): NS = 1 (BF16) or 2 (the split
// residual's hi and lo terms); NP = RHS panels of 128 per CTA.  With NP = 2
// one B operand (the factor record, from HBM) serves two A operands and two
// accumulators, which halves the per-record single-thread steps (producer
// and MMA issuer) per right-hand side; those steps bound the multiply, so
// every configuration also runs four CTAs (four independent pipelines) per
// SM.  Per CTA: PSTAGES 12 KB page stages, an A ring of RING bytes in slots
// of NP x NS x CK x 256 bytes, TMEM of 128 columns: NREG accumulator
// regions of NP x 64 columns.  Measured for one 128-RHS BF16 multiply of the
// 79k-facet terrain (NP = 1): this 1.32 ms; two 16 KB stages and a 20 KB
// ring 1.37 ms; four 8 KB stages 1.43 ms; 16-row chunks in five slots
// 1.56 ms; super-tiles of 128 rows in one 128-column region 1.49 ms; five
// CTAs with one 64-column region each 1.30 ms; three CTAs per SM or two
// CTAs with deeper buffers 1.6-2.1 ms.  Two panels per CTA: 1.23 ms per
// 128 RHS.
template <int NS, int NP> struct TCfg;
template <> struct TCfg<1, 1> {
    static constexpr int PSTAGES = 3, RING = 16384, CTAS = 4, CK = 32, NREG = 2, TMEM = 128;
};
template <> struct TCfg<1, 2> {
    static constexpr int PSTAGES = 3, RING = 16384, CTAS = 4, CK = 16, NREG = 1, TMEM = 128;
};
template <> struct TCfg<2, 1> {
    static constexpr int PSTAGES = 2, RING = 20480, CTAS = 3, CK = 16, NREG = 2, TMEM = 128;
};
// two panels of the split set: 16 KB slots, so three CTAs per SM fit
template <> struct TCfg<2, 2> {
    static constexpr int PSTAGES = 2, RING = 32768, CTAS = 3, CK = 16, NREG = 1, TMEM = 128;
};
// FP8 E4M3 (kind::f8f6f4, K-major operands): the same bytes per slot as BF16
template <> struct TCfg<3, 1> {
    static constexpr int PSTAGES = 3, RING = 16384, CTAS = 4, CK = 64, NREG = 2, TMEM = 128;
};
template <> struct TCfg<3, 2> {
    static constexpr int PSTAGES = 3, RING = 16384, CTAS = 4, CK = 32, NREG = 1, TMEM = 128;
};
// A page set's element kind: S = 1 BF16; S = 2 each FP32 value as two BF16
// terms (hi, lo); S = 3 FP8 E4M3.  terms per element, bytes per term, the K
// of one MMA (records' K granularity) and the alignment of an A operand's
// first panel row (one core-matrix group: 8 rows MN-major BF16; FP8 records
// start on a whole MMA step of 32 rows).
__host__ __device__ constexpr int set_terms(int S) { return S == 2 ? 2 : 1; }
__host__ __device__ constexpr int set_es(int S) { return S == 3 ? 1 : 2; }
__host__ __device__ constexpr int set_kg(int S) { return S == 3 ? 32 : 16; }
__host__ __device__ constexpr int set_al(int S) { return S == 3 ? 32 : 8; }
// record body bytes
__host__ __device__ constexpr int set_body(int S, int K, int N) { return set_terms(S) * set_es(S) * K * N; }
// Shared by every configuration of a page set (records do not depend on NP):
constexpr int kRegion = 64;     // accumulator columns per panel: a phase-1 group's rank columns, a tile's rows
constexpr int kMaxPStages = 4;
template <int NS> __host__ __device__ constexpr int kmax_of() { return NS == 1 ? 64 : NS == 2 ? 32 : 128; }  // K rows per record
// A operands stream through the ring one K chunk of CK rows (all panels and
// terms) per slot, so the copy of one record's later chunks (and of the next
// record) overlaps the MMAs of its earlier ones.
template <int NS, int NP> struct TSlots {
    static constexpr int CK = TCfg<NS, NP>::CK;
    static constexpr int TERM = CK * 128 * set_es(NS);  // one panel, one term
    static constexpr int BYTES = NP * set_terms(NS) * TERM;
    static constexpr int NSLOT = TCfg<NS, NP>::RING / BYTES;
    static_assert(NSLOT >= 2 && NSLOT <= kMaxSlots, "A ring slots");
    static_assert(NP * kRegion * TCfg<NS, NP>::NREG <= TCfg<NS, NP>::TMEM, "accumulator regions");
};
// CTAs of a page set's launches (every configuration of the set has room for them on each SM)
static int cfg_ctas(int S) { return S == 1 ? TCfg<1, 1>::CTAS : S == 2 ? TCfg<2, 2>::CTAS : TCfg<3, 1>::CTAS; }
static int cfg_region(int) { return kRegion; }
static int cfg_kmax(int S) { return S == 1 ? kmax_of<1>() : S == 2 ? kmax_of<2>() : kmax_of<3>(); }
static int cfg_r2(int) { return kRegion; }  // phase-2 (super-)tiles: one row tile
template <int NS, int NP>
constexpr size_t tsmem_bytes() {
    return (size_t)TCfg<NS, NP>::PSTAGES * kTP + TCfg<NS, NP>::RING + 1024;
}
constexpr uint32_t kTWait = 1u << 22;
// record flags: FIRST / LAST record of its accumulator region's use (a
// phase-2 tile, a phase-1 group of units); USTART: first record of a unit
// (its first MMA overwrites D instead of accumulating)
enum { TR_FIRST = 1, TR_LAST = 2, TR_USTART = 4 };
enum { TREC_DENSE = 0, TREC_CSR = 1, TREC_SVDU = 2, TREC_VT = 3, TREC_EMPTY = 4 };

// ------------------------------------------------------------ plan
struct TRec {        // where one tensor record's B operand comes from (build time)
    int32_t kind, blk;
    int32_t K16, N16;
    int32_t row_base;  // absolute tree row of B column 0 (phase 2) -- unused for V'
    int32_t rs, re;    // absolute rows of the block inside this record (phase 2)
    int32_t k0;        // absolute column (phase 2 dense / CSR, phase 1) of B row 0
    int32_t coloff;    // D column offset (phase 2)
    int32_t a_src, a_row0;
    int32_t flags, offT;
    int32_t S;         // 1: BF16 body; 2: hi and lo bodies
    int32_t ring;      // unused (0)
    int32_t dep;       // unused (0)
    int32_t n0;        // V' fills: first rank index of this block's columns
    int32_t nsub;      // V' fills: how many of the block's rank columns
    int32_t bcol;      // V' fills: their first column in the record's B
    int32_t hdr;       // 1: this entry starts a page record (writes its header); 0: another fill of it
    int32_t pad2;
    int64_t dst;
};

}  // namespace vf

// One set of tensor pages: S = 1 holds the BF16 factors; S = 2 holds each
// FP32 factor split in two BF16 terms (hi = bf16(v), lo = bf16(v - hi)),
// two B bodies per record.
struct vf_tensor_set {
    bool built = false;
    int32_t ncta2 = 0, ncta1 = 0;
    vf::dbuf<unsigned char> pages2, pages1;
    vf::dbuf<uint32_t> used2, used1;
    vf::dbuf<int32_t> cta_pages2, cta_pages1;  // ncta + 1 each
    vf::dbuf<int32_t> cta_tiles, cta_tile_ptr; // phase 2: each CTA's (super-)tiles in order
    vf::dbuf<int32_t> st_first, st_count;      // phase 2: rows of each (super-)tile
    vf::dbuf<int32_t> seg_part0;               // phase 2: first (super-)tile of each segment (nseg + 1)
    int64_t nst = 0;                           // (super-)tiles
    vf::dbuf<int32_t> cta_units, cta_unit_ptr; // phase 1: each CTA's units (T row, columns, region column, group end)
    int64_t bytes2 = 0, bytes1 = 0;
    int64_t kind_bytes[5] = {0, 0, 0, 0, 0};   // record bytes by the kind of their first fill
};

struct vf_tensor_plan {
    int64_t n_rows_x = 0, n_rows_t = 0;  // panel rows (X, T), multiples of 16
    std::vector<int32_t> h_offT;         // per block: first T row (SVD), else -1
    // FP8 (S = 3): T rows with each row cluster's run starting on 32 rows,
    // and the static scales (powers of two) that keep every FP8 operand in
    // range: per T row, V' column scale cv and T store scale ct (g = cv ct);
    // per tree row, rs for the phase-2 factors of that row (and 1 / rs)
    int64_t n_rows_t8 = 0;
    std::vector<int32_t> h_offT8;
    vf::dbuf<int32_t> offT8;
    vf::dbuf<float> cv8, ct8, g8, rs8, irs8;
    bool scales8 = false;
    vf_tensor_set set[3];                // [S - 1]
};

namespace vf {

void tensor_plan_free(vf_tensor_plan* p) { delete p; }

// B element (k, mn): the BF16 value, or (S = 2) hi and lo in two bodies `lo_off` bytes apart
__device__ __forceinline__ void st_bf16(unsigned char* base, int64_t k, int mn, int lbo, float v, int lo_off) {
    const int64_t o = (k >> 3) * lbo + (mn >> 3) * 128 + (k & 7) * 16 + (mn & 7) * 2;
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    *reinterpret_cast<__nv_bfloat16*>(base + o) = hi;
    if (lo_off) *reinterpret_cast<__nv_bfloat16*>(base + lo_off + o) = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// The FP8 set's static scales (all NULL for the BF16 sets).
struct F8Scales {
    const float* rs;       // per tree row: phase-2 factors of the row
    const float* g;        // per FP8 T row: cv ct (divides U' columns)
    const float* cv;       // per FP8 T row: V' column scale
    const int32_t* offT8;  // per block: first FP8 T row (SVD), else -1
};

// B element (k, mn) of an FP8 record: K-major core matrices of 8 MN rows x
// 16 K bytes, 16-K groups (N16 / 8) x 128 bytes apart
__device__ __forceinline__ void st_fp8(unsigned char* base, int64_t k, int mn, int n16, float v) {
    const int64_t o = (k >> 4) * (n16 * 16) + (mn >> 3) * 128 + (mn & 7) * 16 + (k & 15);
    base[o] = (unsigned char)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

// One CTA per record: header, zero-filled B body, then the values.
__global__ void k_tpack(const TRec* __restrict__ recs, const HBlock* __restrict__ blocks,
                        const float* __restrict__ val, const int32_t* __restrict__ aux, F8Scales f8,
                        unsigned char* __restrict__ pool) {
    const TRec r = recs[blockIdx.x];
    unsigned char* dst = pool + r.dst;
    uint32_t* h = reinterpret_cast<uint32_t*>(dst);
    if (threadIdx.x == 0 && r.hdr) {
        h[0] = (uint32_t)r.K16;
        h[1] = (uint32_t)r.N16;
        h[2] = (uint32_t)r.coloff;
        h[3] = (uint32_t)r.a_src;
        h[4] = (uint32_t)r.a_row0;
        h[5] = (uint32_t)r.flags;
        h[6] = (uint32_t)r.ring;
        h[7] = (uint32_t)r.dep;
    }
    unsigned char* B = dst + kTRHdr;
    const int lbo = (r.N16 / 8) * 128;
    const int lo = r.S == 2 ? r.K16 * r.N16 * 2 : 0;
    // the pool was cleared: B is zero wherever no fill writes
    if (r.kind == TREC_EMPTY) return;  // a tile with no blocks: a zero product
    const HBlock b = blocks[r.blk];
    if (r.kind == TREC_DENSE) {
        // rows [rs, re) of the block (its part in one row tile: a column-major
        // slab at (rs - r0) * n in the pool), columns [max(k0, c0), min(k0 + K16, c0 + n))
        const int c_lo = max(r.k0, b.c0), c_hi = min(r.k0 + r.K16, b.c0 + b.n);
        const int nr = r.re - r.rs, nc = c_hi - c_lo;
        const float* slab = val + b.off_val + (int64_t)(r.rs - b.r0) * b.n;
        for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
            const int j = e / nr, i = e - j * nr;
            const int row = r.rs + i, col = c_lo + j;
            const float v = slab[(int64_t)(col - b.c0) * nr + i];
            if (r.S == 3) st_fp8(B, col - r.k0, row - r.row_base, r.N16, v * f8.rs[row]);
            else st_bf16(B, col - r.k0, row - r.row_base, lbo, v, lo);
        }
    } else if (r.kind == TREC_CSR) {
        const int32_t* rp = aux + b.off_aux;
        const int32_t* ci = aux + b.off_aux + b.m + 1;
        for (int row = r.rs + (threadIdx.x >> 5); row < r.re; row += blockDim.x >> 5) {
            const int lr = row - b.r0;
            for (int z = rp[lr] + (threadIdx.x & 31); z < rp[lr + 1]; z += 32) {
                const int col = ci[z];
                if (col >= r.k0 && col < r.k0 + r.K16) {
                    if (r.S == 3) st_fp8(B, col - r.k0, row - r.row_base, r.N16, val[b.off_val + z] * f8.rs[row]);
                    else st_bf16(B, col - r.k0, row - r.row_base, lbo, val[b.off_val + z], lo);
                }
            }
        }
    } else if (r.kind == TREC_SVDU) {
        // U' rows (compacted, sorted) inside [rs, re); B row k - k0 holds rank
        // index k, for k in [k0, k0 + K16) (k0 < 0 when the block's T rows
        // start inside the record)
        const int32_t* rows = aux + b.off_aux;
        for (int e = threadIdx.x; e < b.m1 * b.q; e += blockDim.x) {
            const int u = e / b.q, k = e - u * b.q;
            const int row = rows[u];
            if (row >= r.rs && row < r.re && k >= r.k0 && k < r.k0 + r.K16) {
                const float v = val[b.off_val + (int64_t)u * b.q + k];
                if (r.S == 3) st_fp8(B, k - r.k0, row - r.row_base, r.N16, v * f8.rs[row] / f8.g[f8.offT8[r.blk] + k]);
                else st_bf16(B, k - r.k0, row - r.row_base, lbo, v, lo);
            }
        }
    } else {
        // V' rows (compacted columns) inside [k0, k0 + K16); N = the rank
        const int32_t* cols = aux + b.off_aux + b.m1;
        const float* Vp = val + b.off_val + (int64_t)b.m1 * b.q;
        for (int e = threadIdx.x; e < b.n1 * b.q; e += blockDim.x) {
            const int j = e / b.q, k = e - j * b.q;
            const int col = cols[j];
            if (col >= r.k0 && col < r.k0 + r.K16 && k >= r.n0 && k < r.n0 + r.nsub) {
                const float v = Vp[(int64_t)j * b.q + k];
                if (r.S == 3) st_fp8(B, col - r.k0, r.bcol + k - r.n0, r.N16, v * f8.cv[f8.offT8[r.blk] + k]);
                else st_bf16(B, col - r.k0, r.bcol + k - r.n0, lbo, v, lo);
            }
        }
    }
}

__global__ void k_tpage_headers(const int32_t* __restrict__ nrec, const uint32_t* __restrict__ used, int64_t np,
                                unsigned char* __restrict__ pool) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= np) return;
    uint32_t* h = reinterpret_cast<uint32_t*>(pool + p * (int64_t)kTP);
    h[0] = (uint32_t)nrec[p];
    h[1] = used[p];
    h[2] = 0u;
    h[3] = 0u;
}

// ---- FP8 scales (powers of two, so scaling is exact)
// The largest 2^e (|e| <= 126) with v 2^e <= lim, for v > 0 (1 for v not
// finite).  The first guess from log2 is off by at most one either way;
// the two corrections are bounded loops.
__device__ __forceinline__ float pow2_below(float lim, float v) {
    if (!(v > 0.f) || !(v <= 3.0e38f)) return 1.f;
    const float r = lim / v;
    int e = r <= 3.0e38f ? (int)floorf(log2f(r)) : 126;
    e = max(-126, min(e, 126));
    float s = ldexpf(1.f, e);
    for (int i = 0; i < 4 && v * s > lim && s > 1e-37f; ++i) s *= 0.5f;
    for (int i = 0; i < 4 && v * (2.f * s) <= lim && s < 1e37f; ++i) s *= 2.f;
    return s;
}

// Per SVD block (one warp), per rank column t of V': cv scales the column
// to at most 448; ct scales T = (sx X) V' cv back into FP8 range whatever X
// (|T| <= 448 cv ||V'_t||_1 when |sx X| <= 448); g = cv ct.
__global__ void k_f8_vscale(const int32_t* __restrict__ svd, int64_t nsvd, const HBlock* __restrict__ blocks,
                            const float* __restrict__ val, const int32_t* __restrict__ offT8, float* __restrict__ cv,
                            float* __restrict__ ct, float* __restrict__ g) {
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= nsvd) return;
    const int32_t bi = svd[i];
    const HBlock b = blocks[bi];
    const float* Vp = val + b.off_val + (int64_t)b.m1 * b.q;
    for (int t = lane; t < b.q; t += 32) {
        float vmax = 0.f, l1 = 0.f;
        for (int j = 0; j < b.n1; ++j) {
            const float a = fabsf(Vp[(int64_t)j * b.q + t]);
            vmax = fmaxf(vmax, a);
            l1 += a;
        }
        const float c = vmax > 0.f ? pow2_below(448.f, vmax) : 1.f;
        const float d = l1 > 0.f ? pow2_below(1.f, c * l1) : 1.f;
        const int64_t o = offT8[bi] + t;
        cv[o] = c;
        ct[o] = d;
        g[o] = c * d;
    }
}

// Per tree row, the largest phase-2 FP8 operand entry before the row
// scale: dense and CSR entries, U' entries / g.  items: (block, first row,
// end row) -- a dense block once per row tile (its values sit in one
// column-major slab per tile), CSR and SVD blocks once.
__global__ void k_f8_rowmax(const int3* __restrict__ items, int64_t nitems, const HBlock* __restrict__ blocks,
                            const float* __restrict__ val, const int32_t* __restrict__ aux,
                            const float* __restrict__ g8, const int32_t* __restrict__ offT8,
                            unsigned* __restrict__ rowmax) {
    const int64_t it = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (it >= nitems) return;
    const int3 e = items[it];
    const HBlock b = blocks[e.x];
    if (b.kind == VF_BLK_DENSE) {
        const int nr = e.z - e.y;
        const float* slab = val + b.off_val + (int64_t)(e.y - b.r0) * b.n;
        for (int i = lane; i < nr; i += 32) {
            float mx = 0.f;
            for (int j = 0; j < b.n; ++j) mx = fmaxf(mx, fabsf(slab[(int64_t)j * nr + i]));
            atomicMax(rowmax + e.y + i, __float_as_uint(mx));
        }
    } else if (b.kind == VF_BLK_CSR) {
        const int32_t* rp = aux + b.off_aux;
        for (int lr = lane; lr < b.m; lr += 32) {
            float mx = 0.f;
            for (int z = rp[lr]; z < rp[lr + 1]; ++z) mx = fmaxf(mx, fabsf(val[b.off_val + z]));
            atomicMax(rowmax + b.r0 + lr, __float_as_uint(mx));
        }
    } else if (b.kind == VF_BLK_SVD) {
        const int32_t* rows = aux + b.off_aux;
        const int64_t o = offT8[e.x];
        for (int u = lane; u < b.m1; u += 32) {
            float mx = 0.f;
            for (int t = 0; t < b.q; ++t) mx = fmaxf(mx, fabsf(val[b.off_val + (int64_t)u * b.q + t]) / g8[o + t]);
            atomicMax(rowmax + rows[u], __float_as_uint(mx));
        }
    }
}

__global__ void k_f8_rs(const unsigned* __restrict__ rowmax, int64_t n, float* __restrict__ rs,
                        float* __restrict__ irs) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float mx = __uint_as_float(rowmax[i]);
    const float s = mx > 0.f ? pow2_below(448.f, mx) : 1.f;
    rs[i] = s;
    irs[i] = 1.f / s;
}

__global__ void k_fill1(float* __restrict__ a, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) a[i] = 1.f;
}

static vf_status tensor_fp8_scales(vf_hmat* H) {
    vf_tensor_plan* P = H->tplan;
    if (P->scales8) return VF_OK;
    const std::vector<HBlock>& B = H->h_blocks;
    const int64_t nt8 = P->n_rows_t8, n = H->nf;
    VF_TRY(P->offT8.upload(P->h_offT8));
    VF_TRY(P->cv8.alloc(nt8));
    VF_TRY(P->ct8.alloc(nt8));
    VF_TRY(P->g8.alloc(nt8));
    VF_TRY(P->rs8.alloc(std::max<int64_t>(n, 1)));
    VF_TRY(P->irs8.alloc(std::max<int64_t>(n, 1)));
    for (float* a : {P->cv8.p, P->ct8.p, P->g8.p}) k_fill1<<<(unsigned)ceil_div(nt8, 256), 256>>>(a, nt8);
    VF_TRY_CUDA(cudaGetLastError());
    std::vector<int32_t> svd;
    std::vector<int3> items;
    std::vector<int32_t> tile_of_row(n, 0);
    for (size_t k = 0; k < H->h_tile_first.size(); ++k)
        for (int32_t r = H->h_tile_first[k]; r < H->h_tile_first[k] + H->h_tile_count[k]; ++r)
            tile_of_row[r] = (int32_t)k;
    for (size_t bi = 0; bi < B.size(); ++bi) {
        const HBlock& b = B[bi];
        if (b.kind == VF_BLK_SVD) {
            svd.push_back((int32_t)bi);
            items.push_back(make_int3((int)bi, b.r0, b.r0 + b.m));
        } else if (b.kind == VF_BLK_CSR) {
            items.push_back(make_int3((int)bi, b.r0, b.r0 + b.m));
        } else if (b.kind == VF_BLK_DENSE) {
            for (int32_t r = b.r0; r < b.r0 + b.m;) {
                const int32_t k = tile_of_row[r];
                const int32_t re = std::min(b.r0 + b.m, H->h_tile_first[k] + H->h_tile_count[k]);
                items.push_back(make_int3((int)bi, r, re));
                r = re;
            }
        }
    }
    dbuf<int32_t> dsvd;
    dbuf<int3> ditems;
    dbuf<unsigned> rowmax;
    VF_TRY(rowmax.alloc(std::max<int64_t>(n, 1)));
    VF_TRY_CUDA(cudaMemset(rowmax.p, 0, std::max<int64_t>(n, 1) * sizeof(unsigned)));
    if (!svd.empty()) {
        VF_TRY(dsvd.upload(svd));
        k_f8_vscale<<<(unsigned)ceil_div((int64_t)svd.size() * 32, 256), 256>>>(
            dsvd.p, (int64_t)svd.size(), H->blocks.p, H->val.p, P->offT8.p, P->cv8.p, P->ct8.p, P->g8.p);
        VF_TRY_CUDA(cudaGetLastError());
    }
    if (!items.empty()) {
        VF_TRY(ditems.upload(items));
        k_f8_rowmax<<<(unsigned)ceil_div((int64_t)items.size() * 32, 256), 256>>>(
            ditems.p, (int64_t)items.size(), H->blocks.p, H->val.p, H->aux.p, P->g8.p, P->offT8.p, rowmax.p);
        VF_TRY_CUDA(cudaGetLastError());
    }
    if (n > 0) {
        k_f8_rs<<<(unsigned)ceil_div(n, 256), 256>>>(rowmax.p, n, P->rs8.p, P->irs8.p);
        VF_TRY_CUDA(cudaGetLastError());
    }
    VF_TRY_CUDA(cudaDeviceSynchronize());
    P->scales8 = true;
    return VF_OK;
}

// Longest-processing-time assignment of items (costs) to ncta lists.
static std::vector<std::vector<int32_t>> lpt(const std::vector<int64_t>& cost, int32_t ncta) {
    std::vector<int32_t> ord(cost.size());
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
    using Slot = std::pair<int64_t, int32_t>;
    std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
    for (int32_t c = 0; c < ncta; ++c) heap.push({0, c});
    std::vector<std::vector<int32_t>> lists(ncta);
    for (int32_t i : ord) {
        Slot s = heap.top();
        heap.pop();
        lists[s.second].push_back(i);
        s.first += cost[i];
        heap.push(s);
    }
    return lists;
}

// Pack records (grouped: each group starts a new page) into pages per CTA.
static vf_status pack_pages(vf_hmat* H, std::vector<TRec>& recs, const std::vector<std::vector<int32_t>>& cta_groups,
                            const std::vector<std::pair<int64_t, int64_t>>& group_recs, dbuf<unsigned char>& pool,
                            dbuf<uint32_t>& used_d, dbuf<int32_t>& cta_pages, int64_t* bytes,
                            int64_t* kind_bytes, const F8Scales& f8) {
    const int32_t ncta = (int32_t)cta_groups.size();
    std::vector<int32_t> cp(ncta + 1, 0);
    std::vector<uint32_t> used;
    std::vector<int32_t> nrec;
    std::vector<TRec> ordered;
    for (int32_t c = 0; c < ncta; ++c) {
        cp[c] = (int32_t)used.size();
        for (int32_t gi : cta_groups[c]) {
            bool fresh = true;
            for (int64_t ri = group_recs[gi].first; ri < group_recs[gi].second; ++ri) {
                TRec r = recs[ri];
                if (!r.hdr) {  // another fill of the previous record
                    r.dst = ordered.back().dst;
                    ordered.push_back(r);
                    continue;
                }
                const uint32_t sz = (uint32_t)(kTRHdr + set_body(r.S, r.K16, r.N16));
                kind_bytes[r.kind] += sz;
                if (fresh || used.back() + sz > (uint32_t)kTP) {
                    used.push_back(kTPHdr);
                    nrec.push_back(0);
                    fresh = false;
                }
                r.dst = (int64_t)(used.size() - 1) * kTP + used.back();
                used.back() += sz;
                nrec.back()++;
                ordered.push_back(r);
            }
        }
    }
    cp[ncta] = (int32_t)used.size();
    const int64_t np = (int64_t)used.size();
    VF_TRY(pool.alloc(std::max<int64_t>(np, 1) * kTP));
    VF_TRY_CUDA(cudaMemset(pool.p, 0, std::max<int64_t>(np, 1) * kTP));
    VF_TRY(used_d.upload(used));
    VF_TRY(cta_pages.upload(cp));
    *bytes = 0;
    for (uint32_t u : used) *bytes += u;
    if (np == 0) return VF_OK;
    dbuf<TRec> dr;
    VF_TRY(dr.upload(ordered));
    dbuf<int32_t> dn;
    VF_TRY(dn.upload(nrec));
    k_tpack<<<(unsigned)ordered.size(), 256>>>(dr.p, H->blocks.p, H->val.p, H->aux.p, f8, pool.p);
    VF_TRY_CUDA(cudaGetLastError());
    k_tpage_headers<<<(unsigned)ceil_div(np, 256), 256>>>(dn.p, used_d.p, np, pool.p);
    VF_TRY_CUDA(cudaGetLastError());
    VF_TRY_CUDA(cudaDeviceSynchronize());
    return VF_OK;
}

static inline int32_t r16(int64_t x) { return (int32_t)((x + 15) / 16 * 16); }

// The invariants every record must meet (checked on the host before upload).
static vf_status check_records(const std::vector<TRec>& recs, int max_col, int64_t rows_x, int64_t rows_t) {
    for (const TRec& r : recs) {
        const bool ok = (r.S == 1 || r.S == 2 || r.S == 3) && r.K16 >= set_kg(r.S) && r.K16 <= cfg_kmax(r.S) &&
                        r.K16 % set_kg(r.S) == 0 && r.N16 >= 16 && r.N16 <= max_col && r.N16 % 16 == 0 &&
                        r.coloff >= 0 && r.coloff % 16 == 0 && r.coloff + r.N16 <= max_col && r.a_row0 >= 0 &&
                        r.a_row0 % set_al(r.S) == 0 && (int64_t)r.a_row0 + r.K16 <= (r.a_src ? rows_t : rows_x) &&
                        kTPHdr + kTRHdr + set_body(r.S, r.K16, r.N16) <= kTP;
        VF_CHECK(ok, VF_E_INVAL,
                 "tensor plan: bad record (kind %d, K %d, N %d, col %d, src %d, row %d)", r.kind, r.K16, r.N16,
                 r.coloff, r.a_src, r.a_row0);
    }
    return VF_OK;
}

// Runs of occupied kg-column chunks (occ[c] != 0), each at most kmax
// columns: (first chunk, chunks).  K ranges with no nonzero in any of a
// record's pieces are not copied or multiplied.
static std::vector<std::pair<int32_t, int32_t>> chunk_runs(const std::vector<char>& occ, int32_t kmax, int32_t kg) {
    std::vector<std::pair<int32_t, int32_t>> out;
    const int32_t n = (int32_t)occ.size(), lim = kmax / kg;
    for (int32_t c = 0; c < n;) {
        if (!occ[c]) {
            ++c;
            continue;
        }
        int32_t e = c;
        while (e < n && occ[e] && e - c < lim) ++e;
        out.push_back({c, e - c});
        c = e;
    }
    return out;
}

// Build one set of tensor pages of a matrix (once, on first use).
vf_status tensor_plan_build(vf_hmat* H, int S) {
    device_guard g(H->device);
    if (!H->tplan) {
        auto P0 = std::make_unique<vf_tensor_plan>();
        P0->n_rows_x = r16(H->nf) + 32;
        // T rows: q per SVD block, packed; the blocks of one row cluster
        // consecutive from an 8-row boundary (phase 2 reads their T rows
        // as one A operand)
        const std::vector<HBlock>& hb = H->h_blocks;
        std::vector<int32_t> svd;
        for (size_t i = 0; i < hb.size(); ++i)
            if (hb[i].kind == VF_BLK_SVD) svd.push_back((int32_t)i);
        std::stable_sort(svd.begin(), svd.end(), [&](int32_t x, int32_t y) {
            if (hb[x].r0 != hb[y].r0) return hb[x].r0 < hb[y].r0;
            if (hb[x].m != hb[y].m) return hb[x].m < hb[y].m;
            return hb[x].c0 < hb[y].c0;
        });
        P0->h_offT.assign(hb.size(), -1);
        int64_t nt = 0;
        for (size_t k = 0; k < svd.size(); ++k) {
            const int32_t i = svd[k];
            if (k == 0 || hb[i].r0 != hb[svd[k - 1]].r0 || hb[i].m != hb[svd[k - 1]].m) nt = (nt + 7) / 8 * 8;
            P0->h_offT[i] = (int32_t)nt;
            nt += hb[i].q;
        }
        P0->n_rows_t = r16(nt) + 32;
        P0->h_offT8.assign(hb.size(), -1);
        nt = 0;
        for (size_t k = 0; k < svd.size(); ++k) {
            const int32_t i = svd[k];
            if (k == 0 || hb[i].r0 != hb[svd[k - 1]].r0 || hb[i].m != hb[svd[k - 1]].m) nt = (nt + 31) / 32 * 32;
            P0->h_offT8[i] = (int32_t)nt;
            nt += hb[i].q;
        }
        P0->n_rows_t8 = (nt + 31) / 32 * 32 + 128;
        H->tplan = P0.release();
    }
    vf_tensor_plan* P = H->tplan;
    vf_tensor_set* T = &P->set[S - 1];
    if (T->built) return VF_OK;
    const int32_t KG = set_kg(S), AL = set_al(S), TB = set_terms(S) * set_es(S);
    auto rkg = [&](int64_t x) { return (int32_t)((x + KG - 1) / KG * KG); };
    const std::vector<int32_t>& offT = S == 3 ? P->h_offT8 : P->h_offT;
    if (S == 3) VF_TRY(tensor_fp8_scales(H));
    const std::vector<HBlock>& B = H->h_blocks;
    std::vector<int32_t> haux;
    if (H->n_aux > 0) VF_TRY(H->aux.download(haux));
    const int64_t n = H->nf;
    const int64_t ntiles = (int64_t)H->h_tile_first.size();
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, H->device) != cudaSuccess || nsm <= 0) nsm = 148;
    const int64_t rec_cost = 2048;  // fixed work of one record, in byte equivalents

    // ---- phase 2: (super-)tiles of consecutive row tiles up to R2 rows; in
    // each, the pieces of dense and CSR blocks with the same column cluster
    // share records (their rows side by side in B, one copy of the X rows per
    // K-chunk); SVD pieces (A = the block's own T rows) get their own records
    const int32_t r2 = cfg_r2(S);
    std::vector<int32_t> stf, stc, st_of_row(n, -1), tile_of_row(n, -1), segp;
    for (int64_t k = 0, sg = 0; k < ntiles; ++k) {
        const int32_t tf = H->h_tile_first[k], tc = H->h_tile_count[k];
        // (super-)tiles never cross a segment (one mesh of a stacked matrix)
        const bool seg_start = sg < H->nseg() && k == H->h_seg_tile0[sg];
        if (seg_start) segp.push_back((int32_t)stf.size()), ++sg;
        if (stf.empty() || stc.back() + tc > r2 || seg_start) {
            stf.push_back(tf);
            stc.push_back(0);
        }
        stc.back() += tc;
        for (int32_t r = tf; r < tf + tc; ++r) st_of_row[r] = (int32_t)stf.size() - 1, tile_of_row[r] = (int32_t)k;
    }
    const int64_t nst = (int64_t)stf.size();
    struct Piece {
        int32_t blk, rs, re;
    };
    std::vector<std::vector<Piece>> dpieces(nst), spieces(nst);
    for (size_t bi = 0; bi < B.size(); ++bi) {
        const HBlock& b = B[bi];
        if (b.kind != VF_BLK_DENSE && b.kind != VF_BLK_CSR && b.kind != VF_BLK_SVD) continue;
        for (int32_t r = b.r0; r < b.r0 + b.m;) {
            // a dense block's values sit in one slab per row tile, so its
            // pieces end at row tiles; the others' at (super-)tiles
            const int32_t k = st_of_row[r];
            int32_t rs = std::max(b.r0, stf[k]), re = std::min(b.r0 + b.m, stf[k] + stc[k]);
            if (b.kind == VF_BLK_DENSE) {
                const int32_t t = tile_of_row[r];
                rs = std::max(b.r0, H->h_tile_first[t]);
                re = std::min(b.r0 + b.m, H->h_tile_first[t] + H->h_tile_count[t]);
            }
            r = re;
            if (b.kind == VF_BLK_SVD) {
                // any of the block's compacted rows in [rs, re)?
                const int32_t* rows = haux.data() + b.off_aux;
                const int32_t* lo = std::lower_bound(rows, rows + b.m1, rs);
                if (lo == rows + b.m1 || *lo >= re) continue;
                spieces[k].push_back(Piece{(int32_t)bi, rs, re});
            } else {
                dpieces[k].push_back(Piece{(int32_t)bi, rs, re});
            }
        }
    }
    std::vector<TRec> recs2;
    std::vector<std::pair<int64_t, int64_t>> tile_recs(nst);
    std::vector<int64_t> tile_cost(nst, 0);
    for (int64_t k = 0; k < nst; ++k) {
        tile_recs[k].first = (int64_t)recs2.size();
        const int64_t first = (int64_t)recs2.size();
        auto add_cost = [&](const TRec& t) {
            tile_cost[k] += (int64_t)TB * ((int64_t)t.K16 * t.N16 + (int64_t)t.K16 * kPanel) + rec_cost;
        };
        // dense / CSR pieces grouped by column cluster
        std::vector<Piece>& dp = dpieces[k];
        std::stable_sort(dp.begin(), dp.end(), [&](const Piece& x, const Piece& y) {
            const HBlock &bx = B[x.blk], &by = B[y.blk];
            return bx.c0 != by.c0 ? bx.c0 < by.c0 : (bx.n != by.n ? bx.n < by.n : x.rs < y.rs);
        });
        for (size_t i = 0; i < dp.size();) {
            size_t j = i;
            int32_t lo = dp[i].rs, hi = dp[i].re;
            while (j < dp.size() && B[dp[j].blk].c0 == B[dp[i].blk].c0 && B[dp[j].blk].n == B[dp[i].blk].n) {
                lo = std::min(lo, dp[j].rs);
                hi = std::max(hi, dp[j].re);
                ++j;
            }
            const HBlock& b0 = B[dp[i].blk];
            const int32_t coloff = ((lo - stf[k]) / 16) * 16;
            const int32_t row_base = stf[k] + coloff;
            const int32_t n16 = r16(hi - row_base);
            const int32_t kmax = std::min<int32_t>(cfg_kmax(S), ((kTP - kTPHdr - kTRHdr) / (n16 * TB)) / KG * KG);
            const int32_t c8 = (b0.c0 / AL) * AL;
            const int32_t ktot = rkg(b0.c0 + b0.n - c8);
            // KG-column chunks holding a nonzero of some piece (dense pieces: all)
            std::vector<char> occ(ktot / KG, 0);
            for (size_t t = i; t < j; ++t) {
                const HBlock& b = B[dp[t].blk];
                if (b.kind == VF_BLK_DENSE) {
                    for (int32_t c = (b.c0 - c8) / KG; c <= (b.c0 + b.n - 1 - c8) / KG; ++c) occ[c] = 1;
                } else {
                    const int32_t* rp = haux.data() + b.off_aux;
                    const int32_t* ci = rp + b.m + 1;
                    for (int32_t r = dp[t].rs; r < dp[t].re; ++r)
                        for (int32_t z = rp[r - b.r0]; z < rp[r - b.r0 + 1]; ++z) occ[(ci[z] - c8) / KG] = 1;
                }
            }
            for (const auto& run : chunk_runs(occ, kmax, KG)) {
                for (size_t t = i; t < j; ++t) {
                    TRec u{};
                    u.kind = B[dp[t].blk].kind == VF_BLK_DENSE ? TREC_DENSE : TREC_CSR;
                    u.blk = dp[t].blk;
                    u.rs = dp[t].rs;
                    u.re = dp[t].re;
                    u.coloff = coloff;
                    u.row_base = row_base;
                    u.N16 = n16;
                    u.k0 = c8 + KG * run.first;
                    u.K16 = KG * run.second;
                    u.a_src = 0;
                    u.a_row0 = u.k0;
                    u.S = S;
                    u.hdr = t == i;
                    recs2.push_back(u);
                    if (u.hdr) add_cost(u);
                }
            }
            i = j;
        }
        // SVD pieces: blocks of one row cluster with adjacent T rows form a
        // run; K = the run's T rows, in chunks, each block's U' rows filling
        // its own K range (B row = T row - the chunk's first)
        std::vector<Piece>& sp = spieces[k];
        std::stable_sort(sp.begin(), sp.end(),
                         [&](const Piece& x, const Piece& y) { return offT[x.blk] < offT[y.blk]; });
        for (size_t i = 0; i < sp.size();) {
            size_t j = i + 1;
            while (j < sp.size() && B[sp[j].blk].r0 == B[sp[i].blk].r0 && B[sp[j].blk].m == B[sp[i].blk].m &&
                   offT[sp[j].blk] == offT[sp[j - 1].blk] + B[sp[j - 1].blk].q)
                ++j;
            TRec t{};
            t.kind = TREC_SVDU;
            t.rs = sp[i].rs;
            t.re = sp[i].re;
            t.coloff = ((t.rs - stf[k]) / 16) * 16;
            t.row_base = stf[k] + t.coloff;
            t.N16 = r16(t.re - t.row_base);
            t.a_src = 1;
            t.S = S;
            const int32_t kmax = std::min<int32_t>(cfg_kmax(S), ((kTP - kTPHdr - kTRHdr) / (t.N16 * TB)) / KG * KG);
            // from the AL-row boundary at or before the run (rows of other
            // blocks there meet zero B rows)
            const int32_t base = offT[sp[i].blk] / AL * AL;
            const int32_t ktot = rkg(offT[sp[j - 1].blk] + B[sp[j - 1].blk].q - base);
            for (int32_t kc = 0; kc < ktot; kc += kmax) {
                const int32_t a0 = base + kc, kk = std::min(kmax, ktot - kc);
                bool head = true;
                for (size_t u = i; u < j; ++u) {
                    const int32_t o = offT[sp[u].blk], q = B[sp[u].blk].q;
                    if (o + q <= a0 || o >= a0 + kk) continue;
                    TRec f = t;
                    f.blk = sp[u].blk;
                    f.K16 = kk;
                    f.a_row0 = a0;
                    f.k0 = a0 - o;  // rank index of B row 0 (negative when the block starts later)
                    f.hdr = head;
                    recs2.push_back(f);
                    if (head) add_cost(f);
                    head = false;
                }
            }
            i = j;
        }
        if ((int64_t)recs2.size() == first) {
            // a (super-)tile with no blocks still needs its epilogue: one empty record
            TRec t{};
            t.kind = TREC_EMPTY;
            t.K16 = KG;
            t.N16 = 16;
            t.rs = t.re = stf[k];
            t.row_base = t.rs;
            t.S = S;
            t.hdr = 1;
            recs2.push_back(t);
        }
        // FIRST on the first record's header entry, LAST on the last record's
        recs2[first].flags |= TR_FIRST;
        int64_t last_hdr = (int64_t)recs2.size() - 1;
        while (!recs2[last_hdr].hdr) --last_hdr;
        recs2[last_hdr].flags |= TR_LAST;
        tile_recs[k].second = (int64_t)recs2.size();
    }
    {
        std::vector<TRec> heads;
        for (const TRec& t : recs2)
            if (t.hdr) heads.push_back(t);
        VF_TRY(check_records(heads, r2, P->n_rows_x, S == 3 ? P->n_rows_t8 : P->n_rows_t));
    }
    T->nst = nst;
    segp.push_back((int32_t)nst);
    VF_CHECK((int32_t)segp.size() == H->nseg() + 1, VF_E_INVAL, "tensor plan: empty segment");
    VF_TRY(T->seg_part0.upload(segp));
    VF_TRY(T->st_first.upload(stf));
    VF_TRY(T->st_count.upload(stc));
    T->ncta2 = (int32_t)std::min<int64_t>((int64_t)nsm * cfg_ctas(S), nst);
    auto lists2 = lpt(tile_cost, T->ncta2);
    {
        std::vector<int32_t> tiles, ptr(T->ncta2 + 1, 0);
        for (int32_t c = 0; c < T->ncta2; ++c) {
            ptr[c] = (int32_t)tiles.size();
            tiles.insert(tiles.end(), lists2[c].begin(), lists2[c].end());
        }
        ptr[T->ncta2] = (int32_t)tiles.size();
        VF_TRY(T->cta_tiles.upload(tiles));
        VF_TRY(T->cta_tile_ptr.upload(ptr));
    }
    const F8Scales f8s = S == 3 ? F8Scales{P->rs8.p, P->g8.p, P->cv8.p, P->offT8.p} : F8Scales{};
    VF_TRY(pack_pages(H, recs2, lists2, tile_recs, T->pages2, T->used2, T->cta_pages2, &T->bytes2, T->kind_bytes,
                      f8s));

    // ---- phase 1: SVD blocks with the same column cluster (the same X rows)
    // form groups whose ranks fit one accumulator region; a group's records
    // are K-chunks over the cluster's column range, each holding all its
    // blocks' V' side by side (one A copy serves the whole group).  A block
    // of rank above the region width becomes several parts.
    struct Part {
        int32_t blk, n0, nsub;  // rank columns [n0, n0 + nsub) of block blk
    };
    std::vector<std::vector<Part>> groups;
    {
        std::vector<int32_t> order;
        for (size_t bi = 0; bi < B.size(); ++bi)
            if (B[bi].kind == VF_BLK_SVD) order.push_back((int32_t)bi);
        std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
            return B[x].c0 != B[y].c0 ? B[x].c0 < B[y].c0 : B[x].n < B[y].n;
        });
        const int32_t region = cfg_region(S);
        for (size_t i = 0; i < order.size();) {
            size_t j = i;
            while (j < order.size() && B[order[j]].c0 == B[order[i]].c0 && B[order[j]].n == B[order[i]].n) ++j;
            std::vector<Part> cur;
            int32_t used_cols = 0;
            for (size_t t = i; t < j; ++t) {
                const int32_t bi = order[t], q = B[bi].q;
                for (int32_t n0 = 0; n0 < q; n0 += region) {
                    const int32_t nsub = std::min(region, q - n0);
                    if (used_cols + nsub > region) {
                        groups.push_back(cur);
                        cur.clear();
                        used_cols = 0;
                    }
                    cur.push_back(Part{bi, n0, nsub});
                    used_cols += nsub;
                }
            }
            if (!cur.empty()) groups.push_back(cur);
            i = j;
        }
    }
    std::vector<TRec> recs1;
    std::vector<std::pair<int64_t, int64_t>> group_recs1;
    std::vector<int64_t> group_cost;
    for (const auto& g : groups) {
        const HBlock& b0 = B[g[0].blk];
        int32_t n16 = 0;
        for (const Part& pt : g) n16 += pt.nsub;
        n16 = r16(n16);  // the parts' columns side by side, padded once
        const int32_t kmax = std::min<int32_t>(cfg_kmax(S), ((kTP - kTPHdr - kTRHdr) / (n16 * TB)) / KG * KG);
        const int32_t c8 = (b0.c0 / AL) * AL;
        const int32_t ktot = rkg(b0.c0 + b0.n - c8);
        const int64_t first = (int64_t)recs1.size();
        int64_t cost = 0;
        // KG-column chunks holding a compacted column of some block of the group
        std::vector<char> occ(ktot / KG, 0);
        for (const Part& pt : g) {
            const HBlock& b = B[pt.blk];
            const int32_t* cols = haux.data() + b.off_aux + b.m1;
            for (int32_t z = 0; z < b.n1; ++z) occ[(cols[z] - c8) / KG] = 1;
        }
        const auto runs = chunk_runs(occ, kmax, KG);
        for (size_t ri = 0; ri < runs.size(); ++ri) {
            const int32_t kc = KG * runs[ri].first, kk = KG * runs[ri].second;
            int32_t bcol = 0;
            for (size_t pi = 0; pi < g.size(); ++pi) {
                TRec t{};
                t.kind = TREC_VT;
                t.blk = g[pi].blk;
                t.k0 = c8 + kc;
                t.K16 = kk;
                t.N16 = n16;
                t.n0 = g[pi].n0;
                t.nsub = g[pi].nsub;
                t.bcol = bcol;
                t.a_src = 0;
                t.a_row0 = t.k0;
                t.S = S;
                t.hdr = pi == 0;
                t.flags = (ri == 0 && pi == 0) ? (TR_FIRST | TR_USTART) : 0;
                if (ri + 1 == runs.size() && pi == 0) t.flags |= TR_LAST;
                recs1.push_back(t);
                bcol += g[pi].nsub;
            }
            cost += (int64_t)TB * ((int64_t)kk * n16 + (int64_t)kk * kPanel) + rec_cost;
        }
        group_recs1.push_back({first, (int64_t)recs1.size()});
        group_cost.push_back(cost);
    }
    {
        std::vector<TRec> heads;
        for (const TRec& t : recs1)
            if (t.hdr) heads.push_back(t);
        VF_TRY(check_records(heads, cfg_region(S), P->n_rows_x, S == 3 ? P->n_rows_t8 : P->n_rows_t));
    }
    T->ncta1 = (int32_t)std::min<int64_t>((int64_t)nsm * cfg_ctas(S), (int64_t)group_cost.size());
    if (T->ncta1 > 0) {
        auto lists1 = lpt(group_cost, T->ncta1);
        // the epilogue's list: per part, T row, columns, region column, 1 if it ends its group
        std::vector<int32_t> units, ptr(T->ncta1 + 1, 0);
        for (int32_t c = 0; c < T->ncta1; ++c) {
            ptr[c] = (int32_t)(units.size() / 4);
            for (int32_t gi : lists1[c]) {
                int32_t col = 0;
                for (size_t pi = 0; pi < groups[gi].size(); ++pi) {
                    const Part& pt = groups[gi][pi];
                    units.push_back(offT[pt.blk] + pt.n0);
                    units.push_back(pt.nsub);
                    units.push_back(col);
                    units.push_back(pi + 1 == groups[gi].size() ? 1 : 0);
                    col += pt.nsub;
                }
            }
        }
        ptr[T->ncta1] = (int32_t)(units.size() / 4);
        VF_TRY(T->cta_units.upload(units));
        VF_TRY(T->cta_unit_ptr.upload(ptr));
        VF_TRY(pack_pages(H, recs1, lists1, group_recs1, T->pages1, T->used1, T->cta_pages1, &T->bytes1,
                          T->kind_bytes, f8s));
    }
    T->built = true;
    return VF_OK;
}

// ------------------------------------------------------------ device helpers
__device__ __forceinline__ uint64_t mma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// kind::f16 instruction descriptor: D F32, A and B BF16, both MN-major, M = 128
__device__ __forceinline__ uint32_t mma_idesc(int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(kPanel >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// kind::f8f6f4 instruction descriptor: D F32, A and B E4M3, both K-major, M = 128
__device__ __forceinline__ uint32_t mma_idesc_f8(int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kPanel >> 4) << 24);
}

__device__ __forceinline__ void mma_f8(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tm_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    __syncwarp();  // .sync.aligned: the whole warp, converged
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tm_zero16(uint32_t taddr) {
    const uint32_t z = 0u;
    __syncwarp();
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
        "r"(z)
        : "memory");
}

__device__ __forceinline__ void tm_wait_st() {
    __syncwarp();
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ bool bwait(uint64_t* bar, uint32_t parity) {
    return mbar_wait(bar, parity, kTWait);
}

// panel element (row, m) in the MN-major tiled layout (128 RHS)
__device__ __forceinline__ int64_t panel_off(int64_t row, int m) {
    return (row >> 3) * 2048 + (m >> 3) * 128 + (row & 7) * 16 + (m & 7) * 2;
}
// FP8 panel element (row, m): K-major, 16 consecutive rows of one RHS in 16 bytes
__device__ __forceinline__ int64_t panel_off8(int64_t row, int m) {
    return (row >> 4) * 2048 + (m >> 3) * 128 + (m & 7) * 16 + (row & 15);
}
__device__ __forceinline__ unsigned char to_e4m3(float v) {
    return (unsigned char)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}
// FP8 panel rows base + j, j in [jlo, jhi), of RHS m: e[j].  A K-major FP8
// panel keeps 16 consecutive rows of one RHS in 16 bytes, so every 4-row
// word wholly inside the range is one 32-bit store; the rest are bytes
// (rows outside the range belong to other blocks or tiles and stay as they are).
__device__ __forceinline__ void st_fp8_rows(unsigned char* P, int64_t base, int m, int jlo, int jhi,
                                            const unsigned char (&e)[16]) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (j < jlo || j >= jhi) continue;
        const int64_t row = base + j;
        const int j0 = j - (int)(row & 3);  // the first j of row's 4-row word
        if (j0 >= jlo && j0 + 4 <= jhi) {
            if (j == j0)
                *reinterpret_cast<uint32_t*>(P + panel_off8(row, m)) =
                    (uint32_t)e[j] | ((uint32_t)e[j + 1 < 16 ? j + 1 : 15] << 8) |
                    ((uint32_t)e[j + 2 < 16 ? j + 2 : 15] << 16) | ((uint32_t)e[j + 3 < 16 ? j + 3 : 15] << 24);
            continue;
        }
        P[panel_off8(row, m)] = e[j];
    }
}

struct TSmem {
    uint64_t page_full[kMaxPStages], page_empty[kMaxPStages], a_full[kMaxSlots], a_empty[kMaxSlots], d_full[2],
        d_empty[2], done;
    uint32_t tmem_base;
    int32_t abort;
    // the producer's window of page sizes (pages used_base .. + 63 of its list),
    // refilled by 64 independent loads, so no page copy waits on a global load
    int32_t used_base;
    uint32_t used_win[64];
};

static_assert(sizeof(TSmem) <= 1024, "barrier block");

// The RHS panels a kernel reads: X (hi, lo) and T (hi, lo), lo only with
// NS = 2; with NP = 2 the second panel's X and T follow at xstride and
// tstride bytes.
struct TPanels {
    const unsigned char* X[2];
    unsigned char* T[2];
    const float* ct8;          // FP8: per T row, the scale of its stored values
    int64_t rows_x, rows_t;
    int64_t xstride, tstride;
    const int* par;            // ping-pong selection (see TEpi): X[0] = Xalt when *par == 1
    const unsigned char* Xalt;
};

// Apply the ping-pong selection of a graph-captured sweep (every thread, at kernel start).
__device__ __forceinline__ void t_select(TPanels& pn) {
    if (pn.par && *pn.par) pn.X[0] = pn.Xalt;
}
__device__ __forceinline__ void t_select(TEpi& ep) {
    if (ep.par && *ep.par) {
        ep.Y = ep.Yalt;
        ep.Bold = ep.Boldalt;
        ep.Xnext = ep.Xnextalt;
    }
}

// Copy page `next` of the CTA's list into its stage once the page that
// stage held before has been consumed (its MMAs completed): with block, a
// bounded wait for that; without, only a test.  Returns 1 if the copy was
// issued, 0 if the stage is still busy, -1 on a timeout, -2 on a bad page.
template <int NS, int NP>
__device__ __forceinline__ int t_page_refill(TSmem& S, unsigned char* stages, const unsigned char* pages,
                                             const uint32_t* used, int pa, int npl, int next, bool block) {
    constexpr int PS = TCfg<NS, NP>::PSTAGES;
    const int s2 = next % PS;
    if (next >= PS) {
        const uint32_t par = (uint32_t)(((next / PS) - 1) & 1);
        if (block) {
            if (!bwait(&S.page_empty[s2], par)) return -1;
        } else if (!mbar_test_wait(&S.page_empty[s2], par)) {
            return 0;
        }
    }
    const int base = next & ~63;
    if (S.used_base != base) {
#pragma unroll 16
        for (int i = 0; i < 64; ++i) S.used_win[i] = used[pa + min(base + i, npl - 1)];
        S.used_base = base;
    }
    const uint32_t bytes = S.used_win[next & 63];
    if (bytes < kTPHdr || bytes > (uint32_t)kTP || (bytes & 15u)) return -2;
    mbar_arrive_expect_tx(&S.page_full[s2], bytes);
    bulk_g2s(stages + s2 * kTP, pages + (int64_t)(pa + next) * kTP, bytes, &S.page_full[s2]);
    return 1;
}

// The producer (warp 0, lane 0): for each record in order, copies its A
// operand (a contiguous panel range, per panel and term) chunk by chunk into
// the slot ring, each slot reused once the MMAs that read it have completed.
// Pages are refilled as soon as their stage frees (tested between chunks),
// so the A copies of one page never wait for the page before it to be
// consumed.
template <int NS, int NP>
__device__ void t_producer(TSmem& S, unsigned char* stages, unsigned char* abuf, const unsigned char* pages,
                           const uint32_t* used, int pa, int pb, const TPanels& pn, int max_col, int* status) {
    using SL = TSlots<NS, NP>;
    constexpr int PS = TCfg<NS, NP>::PSTAGES;
    const int npl = pb - pa;
    int next = 0, chunk = 0, rc = 0;  // next page to copy; CTA-local chunk index
    for (; next < npl && next < PS; ++next)
        if ((rc = t_page_refill<NS, NP>(S, stages, pages, used, pa, npl, next, true)) < 0) goto bad;
    for (int li = 0; li < npl; ++li) {
        for (; next <= li; ++next)
            if ((rc = t_page_refill<NS, NP>(S, stages, pages, used, pa, npl, next, true)) < 0) goto bad;
        const int s = li % PS;
        if (!bwait(&S.page_full[s], (uint32_t)((li / PS) & 1))) goto fail;
        {
            const unsigned char* pg = stages + s * kTP;
            const int nrec = (int)reinterpret_cast<const uint32_t*>(pg)[0];
            const uint32_t pused = reinterpret_cast<const uint32_t*>(pg)[1];
            uint32_t off = kTPHdr;
            for (int i = 0; i < nrec; ++i) {
                const uint4 h0 = *reinterpret_cast<const uint4*>(pg + off);
                const uint4 h1 = *reinterpret_cast<const uint4*>(pg + off + 16);
                const int K16 = (int)h0.x, N16 = (int)h0.y;
                // self-check: shapes, the record inside the page, the A range inside its panel
                if (K16 < set_kg(NS) || K16 > kmax_of<NS>() || (K16 % set_kg(NS)) || N16 < 16 || N16 > max_col ||
                    (N16 & 15) || (int)h0.z + N16 > max_col || off + kTRHdr + (uint32_t)set_body(NS, K16, N16) > pused ||
                    (h1.x % set_al(NS)) || (int64_t)h1.x + K16 > (h0.w ? pn.rows_t : pn.rows_x))
                    goto oob;
                for (int kc = 0; kc < K16; kc += SL::CK, ++chunk) {
                    if (next < npl) {
                        if ((rc = t_page_refill<NS, NP>(S, stages, pages, used, pa, npl, next, false)) < 0) goto bad;
                        next += rc;
                    }
                    const int slot = chunk % SL::NSLOT, use = chunk / SL::NSLOT;
                    if (use >= 1 && !bwait(&S.a_empty[slot], (uint32_t)((use - 1) & 1))) goto fail;
                    const int ck = min(SL::CK, K16 - kc);
                    // panel rows are aligned to whole core-matrix groups: row r starts at r x 128 x es bytes
                    const uint32_t tb = (uint32_t)ck * kPanel * set_es(NS);
                    const int64_t roff = (int64_t)(h1.x + kc) * kPanel * set_es(NS);
                    mbar_arrive_expect_tx(&S.a_full[slot], NP * set_terms(NS) * tb);
                    for (int q = 0; q < NP; ++q)
                        for (int t = 0; t < set_terms(NS); ++t) {
                            const unsigned char* src =
                                h0.w ? pn.T[t] + q * pn.tstride + roff : pn.X[t] + q * pn.xstride + roff;
                            bulk_g2s(abuf + slot * SL::BYTES + (q * set_terms(NS) + t) * SL::TERM, src, tb,
                                     &S.a_full[slot]);
                        }
                }
                off += kTRHdr + (uint32_t)set_body(NS, K16, N16);
            }
        }
        if (S.abort) return;
    }
    return;
bad:
    if (rc == -2) goto oob;
fail:
    atomicCAS(status, 0, (int)VF_E_TIMEOUT);
    atomicExch(&S.abort, 1);
    return;
oob:
    atomicCAS(status, 0, (int)VF_E_OOB);
    atomicExch(&S.abort, 1);
}

// The MMA issuer (warp 1, lane 0).  With NS = 2 each K step is three MMAs,
// A_hi B_hi + A_lo B_hi + A_hi B_lo (the lo x lo term, ~2^-16 of the
// product, is dropped), all into the same FP32 accumulator; with NP = 2 the
// same B operand meets each panel's A in that panel's accumulator columns.
// The accumulator is NREG regions of NP x 64 columns, used in turn.
template <int NS, int NP>
__device__ void t_issuer(TSmem& S, unsigned char* stages, unsigned char* abuf, int pa, int pb, int* status) {
    using SL = TSlots<NS, NP>;
    constexpr int NREG = TCfg<NS, NP>::NREG, REGW = NP * kRegion;
    int chunk = 0, dcount[2] = {0, 0}, d = 0;
    for (int p = pa, li = 0; p < pb; ++p, ++li) {
        const int s = li % TCfg<NS, NP>::PSTAGES;
        if (!bwait(&S.page_full[s], (uint32_t)((li / TCfg<NS, NP>::PSTAGES) & 1))) goto fail;
        {
            const unsigned char* pg = stages + s * kTP;
            const int nr = (int)reinterpret_cast<const uint32_t*>(pg)[0];
            uint32_t off = kTPHdr;
            for (int r = 0; r < nr; ++r) {
                const uint32_t* h = reinterpret_cast<const uint32_t*>(pg + off);
                const int K16 = (int)h[0], N16 = (int)h[1], coloff = (int)h[2], flags = (int)h[5];
                if (flags & TR_FIRST) {
                    if (!bwait(&S.d_empty[d], (uint32_t)(dcount[d] & 1))) goto fail;
                    tm_fence_after();
                }
                const uint32_t dt = S.tmem_base + (uint32_t)(d * REGW + coloff);
                const uint32_t bsa = smem_u32(pg + off + kTRHdr);
                // B: BF16 MN-major (8-row K groups of N16 x 16 bytes) or FP8 K-major
                // (16-column K groups of N16 x 16 bytes); one MMA step spans two groups
                const uint32_t blbo = NS == 3 ? (uint32_t)N16 * 16 : (uint32_t)(N16 / 8) * 128;
                const uint32_t idesc = NS == 3 ? mma_idesc_f8(N16) : mma_idesc(N16);
                const uint32_t blo = (uint32_t)(K16 * N16 * 2);
                constexpr int KG = set_kg(NS);
                for (int kc = 0; kc < K16; kc += SL::CK, ++chunk) {
                    const int slot = chunk % SL::NSLOT;
                    if (!bwait(&S.a_full[slot], (uint32_t)((chunk / SL::NSLOT) & 1))) goto fail;
                    const uint32_t asa = smem_u32(abuf + slot * SL::BYTES);
                    const int ck = min(SL::CK, K16 - kc);
                    for (int kk = 0; kk < ck / KG; ++kk) {
                        const int ks = kc / KG + kk;  // K step within the record
                        const uint64_t bh = mma_desc(bsa + ks * 2 * blbo, blbo, 128);
                        const int acc = (ks == 0 && (flags & TR_USTART)) ? 0 : 1;
#pragma unroll
                        for (int q = 0; q < NP; ++q) {
                            // one step of A: 16 BF16 rows x 256 bytes, or 32 FP8 rows x 128 bytes
                            const uint32_t aq = asa + (uint32_t)(q * set_terms(NS) * SL::TERM + kk * 4096);
                            const uint64_t ah = mma_desc(aq, 2048, 128);
                            const uint32_t dq = dt + (uint32_t)(q * kRegion);
                            if (NS == 3) mma_f8(dq, ah, bh, idesc, acc);
                            else mma_bf16(dq, ah, bh, idesc, acc);
                            if (NS == 2) {
                                mma_bf16(dq, mma_desc(aq + SL::TERM, 2048, 128), bh, idesc, 1);
                                mma_bf16(dq, ah, mma_desc(bsa + blo + ks * 2 * blbo, blbo, 128), idesc, 1);
                            }
                        }
                    }
                    mma_commit(&S.a_empty[slot]);
                }
                if (flags & TR_LAST) {
                    mma_commit(&S.d_full[d]);
                    dcount[d]++;
                    d = NREG == 1 ? 0 : d ^ 1;
                }
                off += kTRHdr + (uint32_t)set_body(NS, K16, N16);
            }
        }
        mma_commit(&S.page_empty[s]);
        if (S.abort) break;
    }
    mma_commit(&S.done);
    return;
fail:
    atomicCAS(status, 0, (int)VF_E_TIMEOUT);
    atomicExch(&S.abort, 1);
    mma_commit(&S.done);
}

// Common prologue: barriers, TMEM allocation, both regions zeroed.
template <int NS, int NP>
__device__ void t_prologue(TSmem& S) {
    constexpr int ncols = TCfg<NS, NP>::TMEM;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int i = 0; i < TCfg<NS, NP>::PSTAGES; ++i) {
            mbar_init(&S.page_full[i], 1);
            mbar_init(&S.page_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&S.d_full[i], 1);
            mbar_init(&S.d_empty[i], 4);
        }
        for (int i = 0; i < kMaxSlots; ++i) {
            mbar_init(&S.a_full[i], 1);
            mbar_init(&S.a_empty[i], 1);
        }
        mbar_init(&S.done, 1);
        S.abort = 0;
        S.used_base = -64;
        mbar_init_fence();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    if (warp >= 2) {
        // zero the accumulator columns (this warp's 32 lanes), then release both regions
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        for (int c = 0; c < ncols; c += 16) tm_zero16(S.tmem_base + lane_base + c);
        tm_wait_st();
        tm_fence_before();
        __syncwarp();
        if ((threadIdx.x & 31) == 0) {
            mbar_arrive(&S.d_empty[0]);
            mbar_arrive(&S.d_empty[1]);
        }
    }
}

// Common epilogue of a CTA: wait for the MMAs, free TMEM.
template <int NS, int NP>
__device__ void t_finish(TSmem& S, int* status) {
    constexpr int ncols = TCfg<NS, NP>::TMEM;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 32) {
        if (!bwait(&S.done, 0)) atomicCAS(status, 0, (int)VF_E_TIMEOUT);
    }
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem_base), "r"(ncols));
    }
}

// Release a region of REGW columns after the epilogue read it (zeroing it
// first when the next use accumulates into it), then arrive.
template <int REGW>
__device__ __forceinline__ void t_release(TSmem& S, int d, bool zero) {
    const int warp = threadIdx.x >> 5;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    if (zero) {
        for (int c = 0; c < REGW; c += 16) tm_zero16(S.tmem_base + lane_base + d * REGW + c);
        tm_wait_st();
    }
    tm_fence_before();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&S.d_empty[d]);
}

// Drain (producer): wait for every copy it may have left in flight.
template <int NS, int NP>
__device__ void t_drain(TSmem& S) {
    for (int s = 0; s < TCfg<NS, NP>::PSTAGES; ++s)
        mbar_wait(&S.page_full[s], 0, 1024), mbar_wait(&S.page_full[s], 1, 1024);
    for (int j = 0; j < TSlots<NS, NP>::NSLOT; ++j)
        mbar_wait(&S.a_full[j], 0, 1024), mbar_wait(&S.a_full[j], 1, 1024);
}

// ------------------------------------------------------------ phase 1
// T panel rows offT .. + nc of each unit = (V'^T X), per RHS panel.
template <int NS, int NP>
__global__ void __launch_bounds__(192, TCfg<NS, NP>::CTAS) k_tphase1(const unsigned char* __restrict__ pages,
                                                        const uint32_t* __restrict__ used,
                                                        const int32_t* __restrict__ cta_pages,
                                                        const int32_t* __restrict__ cta_units,
                                                        const int32_t* __restrict__ cta_unit_ptr, TPanels pn,
                                                        int* __restrict__ status) {
    constexpr int NREG = TCfg<NS, NP>::NREG, REGW = NP * kRegion;
    t_select(pn);
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* stages = smem;
    unsigned char* abuf = smem + TCfg<NS, NP>::PSTAGES * kTP;
    TSmem& S = *reinterpret_cast<TSmem*>(smem + TCfg<NS, NP>::PSTAGES * kTP + TCfg<NS, NP>::RING);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    t_prologue<NS, NP>(S);
    __syncthreads();
    const int pa = cta_pages[blockIdx.x], pb = cta_pages[blockIdx.x + 1];
    if (warp == 0) {
        if (lane == 0) {
            t_producer<NS, NP>(S, stages, abuf, pages, used, pa, pb, pn, kRegion, status);
            if (S.abort) t_drain<NS, NP>(S);
        }
    } else if (warp == 1) {
        if (lane == 0) t_issuer<NS, NP>(S, stages, abuf, pa, pb, status);
    } else {
        const int m = 32 * (warp & 3) + lane;
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        const int u0 = cta_unit_ptr[blockIdx.x], u1 = cta_unit_ptr[blockIdx.x + 1];
        bool open = false;  // inside a group (its region filled)
        // unit descriptors, 32 at a time: lane i holds unit ub + i
        int4 ud = make_int4(0, 0, 0, 0);
        int ub = u0 - 32;
        for (int u = u0, k = 0; u < u1; ++u) {
            if (u - ub >= 32) {
                ub = u;
                if (u + lane < u1) ud = reinterpret_cast<const int4*>(cta_units)[u + lane];
            }
            const int d = NREG == 1 ? 0 : (k & 1);
            if (!open) {
                if (!__all_sync(0xffffffffu, bwait(&S.d_full[d], (uint32_t)((k / NREG) & 1)))) {
                    if (lane == 0) atomicCAS(status, 0, (int)VF_E_TIMEOUT), atomicExch(&S.abort, 1);
                    break;
                }
                tm_fence_after();
                open = true;
            }
            const int offT = __shfl_sync(0xffffffffu, ud.x, u - ub), nc = __shfl_sync(0xffffffffu, ud.y, u - ub);
            const int col = __shfl_sync(0xffffffffu, ud.z, u - ub);
            const bool gend = __shfl_sync(0xffffffffu, ud.w, u - ub) != 0;
#pragma unroll
            for (int q = 0; q < NP; ++q)
                // the unit's columns [col, col + nc) through 16-column loads
                // aligned inside the panel's 64 columns
                for (int b16 = col & ~15; b16 < col + nc; b16 += 16) {
                    float v[16];
                    tm_ld16(S.tmem_base + lane_base + d * REGW + q * kRegion + b16, v);
                    // FP8: the block's 16 T-row scales, one load per lane, shared by shuffles
                    float ctl = 0.f;
                    if (NS == 3) {
                        const int jj = lane & 15;
                        if (b16 + jj >= col && b16 + jj < col + nc) ctl = pn.ct8[offT + b16 + jj - col];
                        unsigned char e[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) e[j] = to_e4m3(v[j] * __shfl_sync(0xffffffffu, ctl, j));
                        // column b16 + j holds T row base + j; 4-row words wholly
                        // inside this unit's rows are one 32-bit store, the rest bytes
                        const int jlo = max(0, col - b16), jhi = min(16, col + nc - b16);
                        const int64_t base = (int64_t)offT + b16 - col;
                        st_fp8_rows(pn.T[0] + q * pn.tstride, base, m, jlo, jhi, e);
                        continue;
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        if (b16 + j < col || b16 + j >= col + nc) continue;
                        const int64_t row = offT + b16 + j - col;
                        const int64_t o = q * pn.tstride + panel_off(row, m);
                        const __nv_bfloat16 hi = __float2bfloat16_rn(v[j]);
                        *reinterpret_cast<__nv_bfloat16*>(pn.T[0] + o) = hi;
                        if (NS == 2)
                            *reinterpret_cast<__nv_bfloat16*>(pn.T[1] + o) =
                                __float2bfloat16_rn(v[j] - __bfloat162float(hi));
                    }
                }
            if (gend) {
                t_release<REGW>(S, d, false);  // each unit's first MMA overwrites its columns
                open = false;
                ++k;
            }
        }
    }
    t_finish<NS, NP>(S, status);
}

// ------------------------------------------------------------ phase 2
template <int NS, int NP>
__global__ void __launch_bounds__(192, TCfg<NS, NP>::CTAS) k_tphase2(const unsigned char* __restrict__ pages,
                                                        const uint32_t* __restrict__ used,
                                                        const int32_t* __restrict__ cta_pages,
                                                        const int32_t* __restrict__ cta_tiles,
                                                        const int32_t* __restrict__ cta_tile_ptr,
                                                        const int32_t* __restrict__ tile_first,
                                                        const int32_t* __restrict__ tile_count, TPanels pn, TEpi ep,
                                                        int* __restrict__ status) {
    constexpr int NREG = TCfg<NS, NP>::NREG, REGW = NP * kRegion;
    t_select(pn);
    t_select(ep);
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* stages = smem;
    unsigned char* abuf = smem + TCfg<NS, NP>::PSTAGES * kTP;
    TSmem& S = *reinterpret_cast<TSmem*>(smem + TCfg<NS, NP>::PSTAGES * kTP + TCfg<NS, NP>::RING);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    t_prologue<NS, NP>(S);
    __syncthreads();
    const int pa = cta_pages[blockIdx.x], pb = cta_pages[blockIdx.x + 1];
    if (warp == 0) {
        if (lane == 0) {
            t_producer<NS, NP>(S, stages, abuf, pages, used, pa, pb, pn, kRegion, status);
            if (S.abort) t_drain<NS, NP>(S);
        }
    } else if (warp == 1) {
        if (lane == 0) t_issuer<NS, NP>(S, stages, abuf, pa, pb, status);
    } else {
        const int m = 32 * (warp & 3) + lane;
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        const int t0 = cta_tile_ptr[blockIdx.x], t1 = cta_tile_ptr[blockIdx.x + 1];
        // (super-)tile descriptors, 32 at a time: lane i holds tile tb + i
        int my_tile = 0, my_tf = 0, my_tc = 0, tb = t0 - 32;
        for (int ti = t0, k = 0; ti < t1; ++ti, ++k) {
            if (ti - tb >= 32) {
                tb = ti;
                if (ti + lane < t1) {
                    my_tile = cta_tiles[ti + lane];
                    my_tf = tile_first[my_tile];
                    my_tc = tile_count[my_tile];
                }
            }
            const int d = NREG == 1 ? 0 : (k & 1);
            if (!__all_sync(0xffffffffu, bwait(&S.d_full[d], (uint32_t)((k / NREG) & 1)))) {
                if (lane == 0) atomicCAS(status, 0, (int)VF_E_TIMEOUT), atomicExch(&S.abort, 1);
                break;
            }
            tm_fence_after();
            const int tile = __shfl_sync(0xffffffffu, my_tile, ti - tb);
            const int tf = __shfl_sync(0xffffffffu, my_tf, ti - tb), tc = __shfl_sync(0xffffffffu, my_tc, ti - tb);
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const int col = ep.p0 + q * kPanel + m;  // RHS column
                const bool live = col < ep.R;
                unsigned char* xnext = ep.Xnext ? ep.Xnext + q * ep.xstride : nullptr;
                // FP8: D = sx(column) rs(row) (F X); undo both
                const float isx = (NS == 3 && live) ? ep.isx[col] : 1.f;
                const float sxn = (NS == 3 && live) ? ep.sx[col] : 1.f;
                double ss = 0.0;
                for (int c0 = 0; c0 < tc; c0 += 16) {
                    float v[16];
                    tm_ld16(S.tmem_base + lane_base + d * REGW + q * kRegion + c0, v);
                    if (NS == 3) {
                        // the 16 rows' 1 / rs: one load per lane, shared by shuffles (whole warp)
                        const float irl = c0 + (lane & 15) < tc ? ep.irs[tf + c0 + (lane & 15)] : 0.f;
#pragma unroll
                        for (int j = 0; j < 16; ++j) v[j] *= isx * __shfl_sync(0xffffffffu, irl, j);
                    }
                    if (!live) continue;
                    unsigned char e8[16] = {};  // FP8 Jacobi: the next panel's bytes of these rows
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        if (c0 + j >= tc) break;
                        const int64_t p = tf + c0 + j;
                        const int64_t o = (int64_t)col * ep.n + p;
                        if (ep.mode == 0) {
                            ep.Y[o] = v[j];
                        } else if (ep.mode == 2) {
                            // residual r = E - B + rho .* y in FP64
                            const double r = (double)ep.E[o] - (double)ep.Bold[o] + (double)ep.rho[p] * (double)v[j];
                            ss += r * r;
                            ep.Y[o] = (float)r;
                        } else {
                            const float bn = ep.E[o] + ep.rho[p] * v[j];
                            const float dd = bn - ep.Bold[o];
                            ss += (double)dd * dd;
                            ep.Y[o] = bn;
                            if (NS == 3) e8[j] = to_e4m3(bn * sxn);
                            else if (xnext)
                                *reinterpret_cast<__nv_bfloat16*>(xnext + panel_off(p, m)) = __float2bfloat16_rn(bn);
                        }
                    }
                    // the tile's rows only (a 4-row word across a tile boundary is written bytewise)
                    if (NS == 3 && ep.mode == 1 && xnext) st_fp8_rows(xnext, (int64_t)tf + c0, m, 0, min(16, tc - c0), e8);
                }
                if (ep.mode != 0 && live) ep.colpart[(int64_t)col * ep.ntiles + tile] = ss;
            }
            t_release<REGW>(S, d, true);
        }
    }
    t_finish<NS, NP>(S, status);
}

// FP32 column-major (tree order, or face order through perm) -> BF16 panel
// (or, with lo != NULL, the hi and lo panels of the two-term split).
__global__ void k_to_panel(const float* __restrict__ src, int64_t ld, const int32_t* __restrict__ perm, int64_t n,
                           int R, int p0, int64_t rows, unsigned char* __restrict__ hi, unsigned char* __restrict__ lo) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // (row, 8-column chunk)
    if (e >= rows * 16) return;
    const int64_t row = e >> 4;
    const int m0 = (int)(e & 15) * 8;
    __align__(16) __nv_bfloat16 vh[8], vl[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int c = p0 + m0 + i;
        float x = 0.f;
        if (row < n && c < R) x = src[(int64_t)c * ld + (perm ? perm[row] : row)];
        vh[i] = __float2bfloat16_rn(x);
        vl[i] = __float2bfloat16_rn(x - __bfloat162float(vh[i]));
    }
    const int64_t o = (row >> 3) * 2048 + (m0 >> 3) * 128 + (row & 7) * 16;
    *reinterpret_cast<uint4*>(hi + o) = *reinterpret_cast<const uint4*>(vh);
    if (lo) *reinterpret_cast<uint4*>(lo + o) = *reinterpret_cast<const uint4*>(vl);
}

// FP32 column-major (tree order, or face order through perm) -> FP8 panel,
// x sx[column]: one thread per (16-row group, RHS), one 16-byte store.
__global__ void k_to_panel8(const float* __restrict__ src, int64_t ld, const int32_t* __restrict__ perm, int64_t n,
                            int R, int p0, int64_t rows, const float* __restrict__ sx, unsigned char* __restrict__ out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // (16-row group, column)
    if (e >= (rows >> 4) * kPanel) return;
    const int64_t g = e >> 7;
    const int m = (int)(e & 127), c = p0 + m;
    __align__(16) unsigned char v[16];
    const float s = c < R ? sx[c] : 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int64_t row = g * 16 + i;
        float x = 0.f;
        if (row < n && c < R) x = src[(int64_t)c * ld + (perm ? perm[row] : row)];
        v[i] = to_e4m3(x * s);
    }
    *reinterpret_cast<uint4*>(out + g * 2048 + (m >> 3) * 128 + (m & 7) * 16) = *reinterpret_cast<const uint4*>(v);
}

// Per column c < R of an FP32 column-major array: sx = the largest power of
// two with sx max|x| <= 448 h (h: headroom for growth, e.g. Jacobi iterates
// of a right-hand side), and 1 / sx.  One CTA per column.
__global__ void __launch_bounds__(256) k_fp8_colscale(const float* __restrict__ src, int64_t ld,
                                                      const int32_t* __restrict__ perm, int64_t n, float h,
                                                      float* __restrict__ sx, float* __restrict__ isx) {
    const int c = blockIdx.x;
    float mx = 0.f;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
        mx = fmaxf(mx, fabsf(src[(int64_t)c * ld + (perm ? perm[i] : i)]));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __shared__ float wm[8];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) mx = fmaxf(mx, wm[w]);
        const float s = mx > 0.f ? pow2_below(448.f * h, mx) : 1.f;
        sx[c] = s;
        isx[c] = 1.f / s;
    }
}

// ------------------------------------------------------------ host entry
template <int NS, int NP>
static cudaError_t tensor_attrs_cfg() {
    cudaError_t e = cudaFuncSetAttribute(k_tphase1<NS, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tsmem_bytes<NS, NP>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_tphase2<NS, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tsmem_bytes<NS, NP>());
    return e;
}

static vf_status tensor_attrs() {
    static bool done = false;
    if (done) return VF_OK;
    cudaError_t e = tensor_attrs_cfg<1, 1>();
    if (e == cudaSuccess) e = tensor_attrs_cfg<1, 2>();
    if (e == cudaSuccess) e = tensor_attrs_cfg<2, 1>();
    if (e == cudaSuccess) e = tensor_attrs_cfg<2, 2>();
    if (e == cudaSuccess) e = tensor_attrs_cfg<3, 1>();
    if (e == cudaSuccess) e = tensor_attrs_cfg<3, 2>();
    VF_TRY_CUDA(e);
    done = true;
    return VF_OK;
}

vf_status tensor_prepare(vf_hmat* H, int S) {
    VF_TRY(tensor_plan_build(H, S));
    VF_TRY(tensor_attrs());
    return VF_OK;
}

int64_t tensor_panel_bytes_x(const vf_hmat* H) { return H->tplan->n_rows_x * kPanel * 2; }
int64_t tensor_panel_bytes_t(const vf_hmat* H) { return H->tplan->n_rows_t * kPanel * 2; }
int64_t tensor_panel_bytes_x8(const vf_hmat* H) { return H->tplan->n_rows_x * kPanel; }
int64_t tensor_panel_bytes_t8(const vf_hmat* H) { return H->tplan->n_rows_t8 * kPanel; }

vf_status tensor_to_panel8(const vf_hmat* H, const float* X, int64_t ld, const int32_t* perm, int R, int p0,
                           const float* sx, unsigned char* out, cudaStream_t st) {
    const int64_t rows = H->tplan->n_rows_x;
    k_to_panel8<<<(unsigned)ceil_div((rows >> 4) * kPanel, 256), 256, 0, st>>>(X, ld, perm, H->nf, R, p0, rows, sx,
                                                                                out);
    VF_TRY_CUDA(cudaGetLastError());
    return VF_OK;
}

vf_status tensor_fp8_colscale(const vf_hmat* H, const float* X, int64_t ld, const int32_t* perm, int R, float headroom,
                              float* sx, float* isx, cudaStream_t st) {
    if (R <= 0) return VF_OK;
    k_fp8_colscale<<<(unsigned)R, 256, 0, st>>>(X, ld, perm, H->nf, headroom, sx, isx);
    VF_TRY_CUDA(cudaGetLastError());
    return VF_OK;
}

const float* tensor_fp8_irs(const vf_hmat* H) { return H->tplan->irs8.p; }
int64_t tensor_page_bytes(const vf_hmat* H, int S) { return H->tplan->set[S - 1].bytes1 + H->tplan->set[S - 1].bytes2; }

vf_status tensor_to_panel(const vf_hmat* H, const float* X, int64_t ld, const int32_t* perm, int R, int p0,
                          unsigned char* hi, unsigned char* lo, cudaStream_t st) {
    const int64_t rows = H->tplan->n_rows_x;
    k_to_panel<<<(unsigned)ceil_div(rows * 16, 256), 256, 0, st>>>(X, ld, perm, H->nf, R, p0, rows, hi, lo);
    VF_TRY_CUDA(cudaGetLastError());
    return VF_OK;
}

template <int NS, int NP>
static void tensor_launch(const vf_tensor_set& T, const TPanels& pn, const TEpi& ep, int* status, cudaStream_t st) {
    if (T.ncta1 > 0)
        k_tphase1<NS, NP><<<(unsigned)T.ncta1, 192, tsmem_bytes<NS, NP>(), st>>>(
            T.pages1.p, T.used1.p, T.cta_pages1.p, T.cta_units.p, T.cta_unit_ptr.p, pn, status);
    k_tphase2<NS, NP><<<(unsigned)T.ncta2, 192, tsmem_bytes<NS, NP>(), st>>>(
        T.pages2.p, T.used2.p, T.cta_pages2.p, T.cta_tiles.p, T.cta_tile_ptr.p, T.st_first.p, T.st_count.p, pn, ep,
        status);
}

// One multiply of np (1 or 2) RHS panels: phase 1 (T panels), then phase 2
// with the epilogue.  The panels' X (and T) buffers follow each other at
// the panel sizes.
vf_status tensor_multiply(const vf_hmat* H, int S, int np, const unsigned char* Xhi, const unsigned char* Xlo,
                          unsigned char* Thi, unsigned char* Tlo, const TEpi& ep, int* status, cudaStream_t st) {
    VF_CHECK((np == 1 || np == 2) && (S == 1 || S == 2 || S == 3), VF_E_INVAL, "tensor multiply: %d panels, S = %d",
             np, S);
    const vf_tensor_plan* P = H->tplan;
    const vf_tensor_set& T = P->set[S - 1];
    TPanels pn{};
    pn.X[0] = Xhi;
    pn.X[1] = Xlo;
    pn.T[0] = Thi;
    pn.T[1] = Tlo;
    pn.rows_x = P->n_rows_x;
    pn.rows_t = S == 3 ? P->n_rows_t8 : P->n_rows_t;
    pn.xstride = S == 3 ? tensor_panel_bytes_x8(H) : tensor_panel_bytes_x(H);
    pn.tstride = S == 3 ? tensor_panel_bytes_t8(H) : tensor_panel_bytes_t(H);
    pn.ct8 = S == 3 ? P->ct8.p : nullptr;
    pn.par = ep.par;
    pn.Xalt = ep.Xalt;
    if (S == 3 && np == 2) tensor_launch<3, 2>(T, pn, ep, status, st);
    else if (S == 3) tensor_launch<3, 1>(T, pn, ep, status, st);
    else if (S == 2 && np == 2) tensor_launch<2, 2>(T, pn, ep, status, st);
    else if (S == 2) tensor_launch<2, 1>(T, pn, ep, status, st);
    else if (np == 2) tensor_launch<1, 2>(T, pn, ep, status, st);
    else tensor_launch<1, 1>(T, pn, ep, status, st);
    VF_TRY_CUDA(cudaGetLastError());
    return VF_OK;
}

int64_t tensor_parts(const vf_hmat* H, int S) { return H->tplan->set[S - 1].nst; }
const int32_t* tensor_seg_parts(const vf_hmat* H, int S) { return H->tplan->set[S - 1].seg_part0.p; }

int tensor_kernels(const vf_hmat* H, int S) { return (H->tplan->set[S - 1].ncta1 > 0 ? 1 : 0) + 1; }

}  // namespace vf

// The tensor pages of a matrix (built here if not yet): bytes per set and by record kind.
extern "C" vf_status vf_hmat_tensor_bytes(const vf_hmat* h, int32_t terms, int64_t* total, int64_t* by_kind) {
    vf::clear_error();
    VF_CHECK(h && total && (terms == 1 || terms == 2 || terms == 3), VF_E_INVAL, "vf_hmat_tensor_bytes: bad argument");
    VF_CHECK(terms == 3 ? h->has_fp8 : h->has_bf16, VF_E_INVAL, "vf_hmat_tensor_bytes: the matrix has no %s copy",
             terms == 3 ? "FP8" : "BF16");
    vf::device_guard g(h->device);
    VF_TRY(vf::tensor_prepare(const_cast<vf_hmat*>(h), terms));
    const vf_tensor_set& T = h->tplan->set[terms - 1];
    *total = T.bytes1 + T.bytes2;
    if (by_kind)
        for (int k = 0; k < 5; ++k) by_kind[k] = T.kind_bytes[k];
    return VF_OK;
}
