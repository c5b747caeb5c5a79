// The compressed view-factor matrix as stored on the device (tree order).
#pragma once

#include "vf_internal.cuh"

namespace vf {

// One stored block (Algorithm 4 output after flattening the hierarchy).
//  dense: val[off_val + r*n + c], row-major m x n
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

// Row-tile work item (32 bytes): the part of one stored block that lies in
// a tile's rows, as one contiguous range of values.
//  dense: cnt = tile rows, w = n, xoff = tree column c0, val = first value
//         (row lr0 of the block); element e is row e / w, column e % w
//  SVD:   cnt = compacted rows of U' in the tile, w = q, xoff = T slot,
//         val = U' row u0, idx = aux offset of the row-id list at u0
//  CSR:   cnt = tile rows, idx = aux offset of the row pointer of row lr0,
//         idx2 = aux offset of the block's column indices, val = block values
struct TileItem {
    int32_t kind;
    int32_t cnt;
    int32_t w;
    int32_t xoff;
    int32_t idx;
    int32_t idx2;
    int64_t val;
    int32_t blk;
    int32_t pad;
};

// Phase-1 work item: V' rows [j0, j1) of an SVD block, one warp.
struct SvdChunk {
    int32_t blk;
    int32_t j0, j1;
    int32_t chunk;   // index of this chunk within its block
    int32_t nchunks; // chunks of the block
    int32_t first;   // slot of the block's first chunk in the partial buffer
};

}  // namespace vf

struct vf_hmat {
    int device = 0;
    int64_t nf = 0;
    double tol = 0;
    int tree_kind = 0;
    // host mirrors
    std::vector<vf::HBlock> h_blocks;
    std::vector<int32_t> h_perm;
    std::vector<int32_t> h_tile_first, h_tile_count;  // per row tile (tree leaf)
    std::vector<int32_t> h_tile_item_ptr;             // ntiles + 1
    std::vector<int32_t> h_tile_order;                // launch order: heaviest tile first
    int64_t n_part_slots = 0;                         // phase-1 partial slots (split blocks)
    std::vector<vf::TileItem> h_items;
    std::vector<vf::SvdChunk> h_chunks;
    std::vector<float> h_scale8;                      // FP8 per-block scale
    int64_t n_val = 0, n_aux = 0, n_T = 0;            // pool sizes (elements); n_T per RHS column
    int32_t max_q = 0;
    int64_t n_hier = 0;
    vf_assemble_stats stats{};
    // device
    vf::dbuf<int32_t> perm;        // tree position -> facet
    vf::dbuf<int32_t> iperm;       // facet -> tree position
    vf::dbuf<vf::HBlock> blocks;
    vf::dbuf<float> val;           // FP32 master payload
    vf::dbuf<__nv_bfloat16> val16; // BF16 copy
    vf::dbuf<__nv_fp8_e4m3> val8;  // FP8 E4M3 copy (val / scale)
    vf::dbuf<float> scale8;        // per block
    vf::dbuf<int32_t> aux;
    vf::dbuf<int32_t> tile_first, tile_count, tile_item_ptr, tile_order;
    vf::dbuf<vf::TileItem> items;
    vf::dbuf<vf::SvdChunk> chunks;
    bool has_bf16 = false, has_fp8 = false;
    int64_t bytes_payload(int prec) const;
    vf_status upload_all();
};
