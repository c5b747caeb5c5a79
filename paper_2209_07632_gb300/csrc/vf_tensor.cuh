// The tensor-core multiply for panels of 128 right-hand sides (vf_tensor.cu).
#pragma once

#include "vf_hmat.cuh"

namespace vf {

constexpr int kTensorPanel = 128;  // right-hand sides per panel
constexpr int kTensorMinR = 16;    // BF16 multiplies with at least this many columns use the tensor cores

// What phase 2's epilogue does with the finished rows of a tile.
struct TEpi {
    int mode;              // 0: Y = F X;  1: Jacobi B' = E + rho .* (F X)
    int64_t n;             // facets (column stride of the FP32 arrays)
    int R, p0;             // total RHS, first RHS of this panel
    float* Y;              // FP32, column-major tree order (mode 0: F X; mode 1: B')
    const float* E;        // mode 1
    const float* rho;      // mode 1
    const float* Bold;     // mode 1: the previous iterate
    unsigned char* Xnext;  // mode 1: the next BF16 panel (or NULL)
    double* colpart;       // mode 1: per (RHS, tile) sum of squared updates
    int64_t ntiles;
};

// Build the tensor pages once and set the kernels' attributes.
vf_status tensor_prepare(vf_hmat* H);
int64_t tensor_panel_bytes_x(const vf_hmat* H);
int64_t tensor_panel_bytes_t(const vf_hmat* H);
int64_t tensor_page_bytes(const vf_hmat* H);
// FP32 column-major X (ld; row k of the panel = X row perm[k], or k) -> BF16 panel of columns [p0, p0 + 128)
vf_status tensor_to_panel(const vf_hmat* H, const float* X, int64_t ld, const int32_t* perm, int R, int p0,
                          unsigned char* panel, cudaStream_t st);
vf_status tensor_multiply(const vf_hmat* H, const unsigned char* Xpanel, unsigned char* Tpanel, const TEpi& ep,
                          int* status, cudaStream_t st);
int tensor_kernels(const vf_hmat* H);

}  // namespace vf
