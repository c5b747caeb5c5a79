// Internal declarations shared by the libvf translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/vf.h"

namespace vf {

// ------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
void clear_error();

#define VF_TRY_CUDA(expr)                                                              \
    do {                                                                               \
        cudaError_t e_ = (expr);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            ::vf::set_error("%s:%d: %s: %s", __FILE__, __LINE__, #expr, cudaGetErrorString(e_)); \
            return e_ == cudaErrorMemoryAllocation ? VF_E_NOMEM : VF_E_CUDA;           \
        }                                                                              \
    } while (0)

#define VF_CHECK(cond, code, ...)                   \
    do {                                            \
        if (!(cond)) {                              \
            ::vf::set_error(__VA_ARGS__);           \
            return code;                            \
        }                                           \
    } while (0)

#define VF_TRY(expr)                        \
    do {                                    \
        vf_status s_ = (expr);              \
        if (s_ != VF_OK) return s_;         \
    } while (0)

// Allocation-failure injection (vf_debug_fail_alloc): true when the
// library's next device allocation is the one armed to fail.
bool inject_alloc_failure();

// RAII device buffer
template <class T>
struct dbuf {
    T* p = nullptr;
    size_t n = 0;
    dbuf() = default;
    dbuf(const dbuf&) = delete;
    dbuf& operator=(const dbuf&) = delete;
    dbuf(dbuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    dbuf& operator=(dbuf&& o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~dbuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    vf_status alloc(size_t count) {
        release();
        if (count == 0) return VF_OK;
        cudaError_t e = inject_alloc_failure() ? cudaErrorMemoryAllocation : cudaMalloc(&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
            return VF_E_NOMEM;
        }
        n = count;
        return VF_OK;
    }
    vf_status upload(const T* h, size_t count) {
        VF_TRY(alloc(count));
        if (count) VF_TRY_CUDA(cudaMemcpy(p, h, count * sizeof(T), cudaMemcpyHostToDevice));
        return VF_OK;
    }
    vf_status upload(const std::vector<T>& v) { return upload(v.data(), v.size()); }
    vf_status download(std::vector<T>& v) const {
        v.resize(n);
        if (n) VF_TRY_CUDA(cudaMemcpy(v.data(), p, n * sizeof(T), cudaMemcpyDeviceToHost));
        return VF_OK;
    }
};

// Scoped device selection
struct device_guard {
    int prev = -1;
    explicit device_guard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~device_guard() {
        int cur;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// ------------------------------------------------------------ BVH
// Axis-aligned boxes in the scale-3 integer frame; leaves hold <= 4
// triangles.  Children of an inner node are stored at `left` and `left+1`.
struct BvhNode {
    int32_t lo[3];
    int32_t hi[3];
    int32_t left;   // inner: first child; leaf: first triangle slot
    int32_t count;  // 0 for inner nodes
};
struct BvhTri {
    int32_t v[9];   // scale-3 vertex coordinates a, b, c
    int32_t facet;  // face index
    int32_t pad[2];
};

// ------------------------------------------------------------ handles
}  // namespace vf

struct vf_mesh {
    int device = 0;
    int64_t nf = 0, nv = 0;
    double unit = 0;
    int64_t base[3] = {0, 0, 0};
    std::vector<int32_t> h_faces;
    // device, face order
    vf::dbuf<int32_t> q;        // nv x 3 grid coordinates
    vf::dbuf<int32_t> faces;    // nf x 3
    vf::dbuf<int32_t> c3;       // nf x 3 : a + b + c
    vf::dbuf<long long> nint;   // nf x 3 : (b-a) x (c-a)
    vf::dbuf<double> area;      // nf
    vf::dbuf<double> cent;      // nf x 3 (relative to the grid origin)
    vf::dbuf<double> nrm;       // nf x 3 unit normals
    // host copies for tree building
    std::vector<int32_t> h_c3;
    // BVH (device)
    vf::dbuf<vf::BvhNode> bvh_nodes;
    vf::dbuf<vf::BvhTri> bvh_tris;
    int32_t bvh_depth = 0;
};

struct vf_tree {
    int kind = 0, leaf_size = 64, max_depth = 32;
    int64_t nf = 0;
    std::vector<int32_t> perm;                   // tree position -> facet
    std::vector<int32_t> first, count, depth, parent;
    std::vector<std::vector<int32_t>> kids;      // child ids in child-index order
    bool is_leaf(int k) const { return kids[k].empty(); }
};

namespace vf {

// ------------------------------------------------------------ shared helpers
vf_status bvh_build(vf_mesh* m);

// visibility bit matrix over an index map (tree order): bits[i * ldw + w],
// ldw = ceil(n / 32) words per row; index[k] = facet at position k.
vf_status visibility_bits(const vf_mesh* m, const int32_t* d_index, int64_t n, uint32_t* d_bits,
                          int64_t ldw, cudaStream_t st);

// counter-based hash -> uniform float in (-1, 1) (SplitMix64 finaliser)
__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

double now_seconds();

}  // namespace vf
