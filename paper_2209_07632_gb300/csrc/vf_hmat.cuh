// The compressed view-factor matrix as stored on the device (tree order).
#pragma once

#include <atomic>
#include <map>
#include <mutex>

#include "vf_internal.cuh"

namespace vf {

// One stored block (Algorithm 4 output after flattening the hierarchy).
//  dense: per row tile [rs, re) the block meets, a column-major slab at
//         val[off_val + (rs - r0)*n]: element (row, c) at
//         (rs - r0)*n + c*(re - rs) + (row - rs)
//  CSR:   aux[off_aux .. +m] row pointers (local), aux[off_aux+m+1 ..] global
//         tree-order column of each nonzero, val[off_val + k]
//  SVD:   aux[off_aux .. +m1] global tree rows, aux[off_aux+m1 .. +n1] global
//         tree columns; U' = val[off_val ..] (m1 x q row-major, Sigma folded
//         in), V' = val[off_val + m1*q ..] (n1 x q row-major)
struct HBlock {
    int32_t kind;
    int32_t I, J;         // tree nodes
    int32_t r0, m, c0, n; // tree-order ranges
    int32_t q, m1, n1;    // SVD rank and compacted sizes (nnz count for CSR in m1)
    int64_t off_val;
    int64_t off_aux;
    int64_t off_T;        // SVD: offset of its q-vector slot in the T buffer (per RHS column)
};

// The multiply streams the matrix from tile-major "pages": kPage-byte
// blocks, built once from the block pools.  A page is one bulk copy into a
// warp's prefetch stage.  Layout:
//   page header (16 B): u32 number of records, u32 bytes used, u32 nx, u32 0
//   x list (nx x i32): where each x value the page's records need comes from
//               (>= 0: a tree-order row of X; < 0: T slot -1 - v); on arrival
//               the warp gathers all of them in one round and overwrites the
//               list with the values, so records compute from shared memory
//   records, 16-byte aligned (from page_rec0(nx)), each padded to 16 bytes:
//   header (16 B): u32 kind | cnt << 8 | roff << 16, u32 w, u32 xbase (first
//               entry in the page's x list), f32 scale
//   dense  (1): cnt x w column-major slab (element (r, k) at k * cnt + r) of
//               tile rows roff..roff+cnt-1; x entries: its w columns
//   CSR    (2): tile rows roff..roff+cnt-1, w = nnz; row pointers (cnt + 1,
//               from 0), values (nnz); x entries: the nonzeros' columns
//   SVD    (3): w = q; tile-local rows (cnt bytes), U' (cnt x q) as a
//               column-major slab; x entries: its q T slots.  The same
//               layout carries a CSR block's piece where that is smaller:
//               its nonempty rows x the columns they use, zeros stored,
//               x entries: those columns (one gather per column instead
//               of one per nonzero)
//   long CSR row (5): tile row roff, w = nnz; values; x entries: columns
//   phase-1 (6): header + i32 chunk (within its unit), chunks in the unit,
//               partial offset (-1: the unit is the whole block), T slot;
//               cnt = rows, w = q; V' rows (cnt x q, row-major); x entries:
//               the rows' columns
#ifndef VF_PAGE_BYTES
#define VF_PAGE_BYTES 4096
#endif
constexpr int kPage = VF_PAGE_BYTES;
constexpr int kPageHdr = 16;
constexpr int kRecHdr = 16;
constexpr int kP1Hdr = 32;
// Every x entry comes with at least 4 bytes of FP32 values in its record,
// so a page planned with FP32 sizes holds fewer than kPage / 8 x entries;
// the planner checks this bound.
constexpr int kXMax = kPage / 8;
enum RecKind { REC_DENSE = 1, REC_CSR = 2, REC_SVD = 3, REC_CSR_LONG = 5, REC_P1 = 6 };

__host__ __device__ inline uint32_t pad4(uint32_t b) { return (b + 3u) & ~3u; }
__host__ __device__ inline uint32_t pad16(uint32_t b) { return (b + 15u) & ~15u; }

// bytes of a record's header and body (not its x entries), element size
// es, padded to 16 so every record header is one vector load
__host__ __device__ inline uint32_t rec_bytes(int kind, int cnt, int w, int es) {
    switch (kind) {
        case REC_DENSE: return pad16(kRecHdr + (uint32_t)(cnt * w * es));
        case REC_SVD: return pad16(kRecHdr + pad4((uint32_t)cnt) + (uint32_t)(cnt * w * es));
        case REC_CSR: return pad16(kRecHdr + 4u * (cnt + 1) + (uint32_t)(w * es));
        case REC_CSR_LONG: return pad16(kRecHdr + (uint32_t)(w * es));
        default: return pad16(kP1Hdr + (uint32_t)(cnt * w * es));
    }
}

// offset of the first record in a page whose x list has nx entries
__host__ __device__ inline uint32_t page_rec0(uint32_t nx) { return kPageHdr + pad16(4u * nx); }

// Planning weight of one record beyond its bytes: the fixed work of
// decoding and finishing it, in byte equivalents of streaming.
constexpr int64_t kRecCost = 384;

// x entries a record adds to its page's x list
__host__ __device__ inline uint32_t rec_xn(int kind, int cnt, int w) {
    return kind == REC_P1 ? (uint32_t)cnt : (uint32_t)w;
}

// Where one record's data comes from in the block pools (build time only).
struct RecSrc {
    int32_t kind, cnt, w, x;
    int32_t blk;
    int32_t roff;        // dense: first tile row of the slab
    int32_t tile_first;  // SVD: row ids are stored relative to it
    int64_t val;         // element offset of the first value in the block pool
    int32_t idx;         // CSR: aux offset of the first row pointer; SVD: of the first row id
    int32_t idx2;        // CSR / long row / phase 1: aux offset of the first column index
    int32_t nz0;         // CSR: block-local offset of the first nonzero
    int32_t chunk, nchunks, first;  // phase 1: chunk in its unit, unit chunks, partial slot or -1
    int64_t dst;         // byte offset of the record in the page pool (per element size)
    int64_t xdst;        // byte offset of its first x-list entry in the page pool
    int32_t xbase;       // its first x-list entry within the page
    int32_t csr;         // REC_SVD layout filled from a CSR block: its nonempty rows x its columns, dense
                         // (rows, then columns, at xtra[idx]; rp at aux[nz0], cols at aux[idx2]; block row first)
};

}  // namespace vf

struct vf_tensor_plan;  // the tensor-core multiply's pages (vf_tensor.cu), built on first use
namespace vf {
void tensor_plan_free(vf_tensor_plan* p);
// a process-unique id per matrix handle (keys of caches built from handles)
inline uint64_t next_hmat_uid() {
    static std::atomic<uint64_t> c{0};
    return ++c;
}
}

struct vf_hmat {
    uint64_t uid = vf::next_hmat_uid();
    // the autotuner's choices per (precision, R): vf_tune records
    mutable std::mutex tune_mu;
    mutable std::map<std::pair<int, int>, vf_tune> tunes;
    int device = 0;
    int64_t nf = 0;
    double tol = 0;
    int tree_kind = 0;
    // host mirrors
    std::vector<vf::HBlock> h_blocks;
    std::vector<int32_t> h_perm;
    std::vector<int32_t> h_tile_first, h_tile_count;  // per row tile (tree leaf)
    std::vector<int32_t> h_tile_page_ptr;             // ntiles * kWarps + 1: each warp's page range
    std::vector<int32_t> h_tile_order;                // launch order: heaviest tile first
    std::vector<int32_t> h_p1_warp_ptr;               // phase 1: each warp's page range (n_p1_warps + 1)
    int64_t n_p1_warps = 0;                           // a multiple of 8 (one CTA per 8 warps)
    int64_t n_pages = 0, n_p1_pages = 0;              // phase-2 / phase-1 pages
    int64_t n_part_slots = 0;                         // phase-1 partial floats per RHS column (cut blocks)
    int64_t n_split = 0;                              // blocks whose V' rows span several records
    int64_t n_val = 0, n_aux = 0, n_T = 0;            // pool sizes (elements); n_T per RHS column
    int32_t max_q = 0;
    int64_t n_hier = 0;
    vf_assemble_stats stats{};
    std::vector<float> h_probe_feat;                  // the probe log: VF_PRED_NFEAT per candidate
    std::vector<int32_t> h_probe_label;               // its outcomes (classes)
    // device: block pools (the stored representation)
    vf::dbuf<int32_t> perm;        // tree position -> facet
    vf::dbuf<int32_t> iperm;       // facet -> tree position
    vf::dbuf<vf::HBlock> blocks;
    vf::dbuf<float> val;           // FP32 master payload
    vf::dbuf<__nv_bfloat16> val16; // BF16 copy
    vf::dbuf<__nv_fp8_e4m3> val8;  // FP8 E4M3 copy (val / scale)
    vf::dbuf<float> scale8;        // per block
    vf::dbuf<int32_t> aux;
    // device: the multiply's page pools per precision (FP32, BF16, FP8)
    vf::dbuf<unsigned char> pages[3], p1pages[3];
    vf::dbuf<uint16_t> page_used[3], p1_used[3];  // bytes used per page
    vf::dbuf<int32_t> tile_first, tile_count, tile_page_ptr, tile_order;
    vf::dbuf<int32_t> p1_split;                       // n_split x {first slot, chunks, q, T slot, block}
    vf::dbuf<int32_t> p1_warp_ptr;
    bool has_bf16 = false, has_fp8 = false;
    vf_tensor_plan* tplan = nullptr;
    // Segments: the meshes of a stacked (block-diagonal) matrix, as row and
    // row-tile ranges (nseg + 1 entries each); a plain matrix is one segment.
    // The solve tracks convergence per segment and column.
    std::vector<int32_t> h_seg_row0, h_seg_tile0;
    vf::dbuf<int32_t> seg_row0, seg_tile0;
    int32_t nseg() const { return h_seg_row0.empty() ? 1 : (int32_t)h_seg_row0.size() - 1; }
    ~vf_hmat() { vf::tensor_plan_free(tplan); }
    int64_t bytes_payload(int prec) const;        // bytes of the stored representation
    vf_status upload_all();
};
