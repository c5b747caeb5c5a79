// The tensor-core multiply for panels of 128 right-hand sides (vf_tensor.cu).
#pragma once

#include "vf_hmat.cuh"

namespace vf {

constexpr int kTensorPanel = 128;  // right-hand sides per panel
constexpr int kTensorMinR = 16;    // BF16 multiplies with at least this many columns use the tensor cores

// What phase 2's epilogue does with the finished rows of a tile.
struct TEpi {
    int mode;              // 0: Y = F X;  1: Jacobi B' = E + rho .* (F X);
                           // 2: residual r = E - B + rho .* (F B) in FP64 (Y = r, colpart = r^2)
    int64_t n;             // facets (column stride of the FP32 arrays)
    int R, p0;             // total RHS, first RHS of this panel
    float* Y;              // FP32, column-major tree order (mode 0: F X; mode 1: B')
    const float* E;        // mode 1
    const float* rho;      // mode 1
    const float* Bold;     // mode 1: the previous iterate; mode 2: B
    unsigned char* Xnext;  // mode 1: the next BF16 (FP8) panel (or NULL); a second panel at + xstride bytes
    int64_t xstride;
    double* colpart;       // modes 1, 2: per (RHS, tile) sums of squares
    int64_t ntiles;
    // FP8 (S = 3): the product is sx(column) rs(row) F X; sx and 1 / sx per
    // RHS column (global index), 1 / rs per tree row.  Xnext is written as
    // FP8 of sx B'.
    const float* sx;
    const float* isx;
    const float* irs;
    // Ping-pong selection for a sweep captured once in a CUDA graph: when
    // par is not NULL and *par (read when the kernel starts) is 1, the
    // kernels use Xalt (the input panel), Yalt, Boldalt and Xnextalt
    // instead of the input panel, Y, Bold and Xnext.
    const int* par;
    const unsigned char* Xalt;
    float* Yalt;
    const float* Boldalt;
    unsigned char* Xnextalt;
};

// Build one page set of the matrix once (S = 1: BF16 factors; S = 2: each
// FP32 factor as two BF16 terms hi + lo; S = 3: FP8 E4M3 factors with
// power-of-two scales per row and per SVD rank column) and set the
// kernels' attributes.
vf_status tensor_prepare(vf_hmat* H, int S);
int64_t tensor_panel_bytes_x(const vf_hmat* H);
int64_t tensor_panel_bytes_t(const vf_hmat* H);
int64_t tensor_page_bytes(const vf_hmat* H, int S);
// FP32 column-major X (ld; panel row k = X row perm[k], or k) -> the BF16
// panel of columns [p0, p0 + 128), and with lo != NULL also the lo panel of
// the two-term split (x = hi + lo + O(2^-16 x))
vf_status tensor_to_panel(const vf_hmat* H, const float* X, int64_t ld, const int32_t* perm, int R, int p0,
                          unsigned char* hi, unsigned char* lo, cudaStream_t st);
// One multiply of np RHS panels (np = 2 only with S = 1; the panels' X and
// T buffers follow each other at the panel sizes).  S = 1: BF16 products;
// S = 2: the split products A_hi B_hi + A_lo B_hi + A_hi B_lo (FP32-factor
// accuracy to ~2^-16).
vf_status tensor_multiply(const vf_hmat* H, int S, int np, const unsigned char* Xhi, const unsigned char* Xlo,
                          unsigned char* Thi, unsigned char* Tlo, const TEpi& ep, int* status, cudaStream_t st);
int tensor_kernels(const vf_hmat* H, int S);
// FP8 (S = 3) panels: 128 bytes per panel row, K-major
int64_t tensor_panel_bytes_x8(const vf_hmat* H);
int64_t tensor_panel_bytes_t8(const vf_hmat* H);
// per column c < R: sx[c] = the largest power of two with sx max|x| <= 448 headroom, isx = 1 / sx
vf_status tensor_fp8_colscale(const vf_hmat* H, const float* X, int64_t ld, const int32_t* perm, int R, float headroom,
                              float* sx, float* isx, cudaStream_t st);
// FP32 column-major X -> the FP8 panel of columns [p0, p0 + 128), scaled by sx per column
vf_status tensor_to_panel8(const vf_hmat* H, const float* X, int64_t ld, const int32_t* perm, int R, int p0,
                           const float* sx, unsigned char* out, cudaStream_t st);
// 1 / rs per tree row (the FP8 set's row scales; after tensor_prepare(H, 3))
const float* tensor_fp8_irs(const vf_hmat* H);
// per-column partial sums a phase-2 epilogue writes (one per row part)
int64_t tensor_parts(const vf_hmat* H, int S);
// first part of each segment (nseg + 1 entries, device)
const int32_t* tensor_seg_parts(const vf_hmat* H, int S);

}  // namespace vf
