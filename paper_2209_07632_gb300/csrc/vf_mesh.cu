// Mesh geometry, Algorithm 2 partition, BVH and exact visibility / insolation.
//
// Geometry (Section 3): A_i, x_i, n_i from vertices snapped to a 2^18 grid.
// Visibility (Section 3.2): back-face cull n_i.d_ij > 0 and n_j.d_ji > 0,
// then an occlusion test of the open segment between the centroids.
// Insolation (Section 2, Eq. insolation-for-point-sun).
//
// Exactness: grid coordinates are < 2^18 + 2; points are handled at scale 3
// (a + b + c = 3 x centroid), so coordinate differences are < 2^19.6 and each
// 3x3 determinant below is < 2^61.8 in magnitude: int64 arithmetic decides
// every predicate exactly, identically on any machine.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <chrono>

#include "vf_internal.cuh"

namespace vf {

static thread_local char g_err[1024] = "";

// vf_debug_fail_alloc: allocations left before the armed one (0: disarmed)
static std::atomic<int64_t> g_fail_alloc{0};

bool inject_alloc_failure() {
    int64_t c = g_fail_alloc.load(std::memory_order_relaxed);
    while (c > 0) {
        if (g_fail_alloc.compare_exchange_weak(c, c - 1, std::memory_order_relaxed)) return c == 1;
    }
    return false;
}

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = 0; }

double now_seconds() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ------------------------------------------------------------ predicates
struct P3 { long long x, y, z; };

__device__ __forceinline__ P3 mk(const int32_t* v) { return P3{v[0], v[1], v[2]}; }
__device__ __forceinline__ P3 sub(P3 a, P3 b) { return P3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ long long det(P3 u, P3 v, P3 w) {
    long long cx = v.y * w.z - v.z * w.y;
    long long cy = v.z * w.x - v.x * w.z;
    long long cz = v.x * w.y - v.y * w.x;
    return u.x * cx + u.y * cy + u.z * cz;
}
__device__ __forceinline__ int sgn(long long x) { return (x > 0) - (x < 0); }

// sign of orient(a,b,c,d) = det[b-a, c-a, d-a]
__device__ __forceinline__ int orient(P3 a, P3 b, P3 c, P3 d) { return sgn(det(sub(b, a), sub(c, a), sub(d, a))); }

// Open segment P-Q against the closed triangle t (scale 3).
__device__ __forceinline__ bool seg_hits(P3 P, P3 Q, const BvhTri& t) {
    P3 A = mk(t.v), B = mk(t.v + 3), C = mk(t.v + 6);
    int s1 = orient(A, B, C, P), s2 = orient(A, B, C, Q);
    if (s1 == 0 || s2 == 0 || s1 == s2) return false;
    int e1 = orient(P, Q, A, B), e2 = orient(P, Q, B, C), e3 = orient(P, Q, C, A);
    return (e1 >= 0 && e2 >= 0 && e3 >= 0) || (e1 <= 0 && e2 <= 0 && e3 <= 0);
}

// Ray P + tD (t > 0) against the closed triangle t.
__device__ __forceinline__ bool ray_hits(P3 P, P3 D, const BvhTri& t) {
    P3 A = mk(t.v), B = mk(t.v + 3), C = mk(t.v + 6);
    P3 u = sub(B, A), w = sub(C, A);
    int s1 = sgn(det(u, w, sub(P, A)));
    // n . D with n = u x w
    long long nx = u.y * w.z - u.z * w.y, ny = u.z * w.x - u.x * w.z, nz = u.x * w.y - u.y * w.x;
    int sd = sgn(nx * D.x + ny * D.y + nz * D.z);
    if (s1 == 0 || sd == 0 || s1 == sd) return false;
    P3 a = sub(A, P), b = sub(B, P), c = sub(C, P);
    int e1 = sgn(det(D, a, b)), e2 = sgn(det(D, b, c)), e3 = sgn(det(D, c, a));
    return (e1 >= 0 && e2 >= 0 && e3 >= 0) || (e1 <= 0 && e2 <= 0 && e3 <= 0);
}

// Conservative slab test: boxes widened by 4 grid units (scale 3); all
// integer inputs are exact in FP32 (< 2^21) and the widening exceeds the
// rounding of the parametric bounds, so a box the exact set meets is never
// rejected.
__device__ __forceinline__ bool box_hit(const BvhNode& nd, float px, float py, float pz, float ix, float iy,
                                        float iz, float tmax) {
    float t0 = 0.f, t1 = tmax;
    float a = (float(nd.lo[0] - 4) - px) * ix, b = (float(nd.hi[0] + 4) - px) * ix;
    t0 = fmaxf(t0, fminf(a, b));
    t1 = fminf(t1, fmaxf(a, b));
    a = (float(nd.lo[1] - 4) - py) * iy;
    b = (float(nd.hi[1] + 4) - py) * iy;
    t0 = fmaxf(t0, fminf(a, b));
    t1 = fminf(t1, fmaxf(a, b));
    a = (float(nd.lo[2] - 4) - pz) * iz;
    b = (float(nd.hi[2] + 4) - pz) * iz;
    t0 = fmaxf(t0, fminf(a, b));
    t1 = fminf(t1, fmaxf(a, b));
    return t0 <= t1;
}

__device__ __forceinline__ float safe_inv(long long d) { return d == 0 ? 1e30f : 1.0f / float(d); }

constexpr int kStack = 64;

// Any-hit query.  mode 0: open segment P->Q skipping facets fi, fj;
// mode 1: ray from P along Q (a direction) skipping facet fi.
template <int MODE>
__device__ bool bvh_blocked(const BvhNode* __restrict__ nodes, const BvhTri* __restrict__ tris, P3 P, P3 Q,
                            int fi, int fj) {
    P3 D = MODE == 0 ? sub(Q, P) : Q;
    float px = float(P.x), py = float(P.y), pz = float(P.z);
    float ix = safe_inv(D.x), iy = safe_inv(D.y), iz = safe_inv(D.z);
    float tmax = MODE == 0 ? 1.0f : 3.0e38f;
    int stack[kStack];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        BvhNode nd = nodes[stack[--sp]];
        if (!box_hit(nd, px, py, pz, ix, iy, iz, tmax)) continue;
        if (nd.count > 0) {
            for (int s = nd.left; s < nd.left + nd.count; ++s) {
                BvhTri t = tris[s];
                if (t.facet == fi || t.facet == fj) continue;
                if (MODE == 0 ? seg_hits(P, Q, t) : ray_hits(P, Q, t)) return true;
            }
        } else if (sp + 2 <= kStack) {
            stack[sp++] = nd.left + 1;
            stack[sp++] = nd.left;
        } else {
            return true;  // unreachable for the median-split depth (< 40); conservative
        }
    }
    return false;
}

__device__ __forceinline__ bool cull_pass(const int32_t* __restrict__ c3, const long long* __restrict__ nint, int i,
                                          int j) {
    long long dx = (long long)c3[3 * j] - c3[3 * i];
    long long dy = (long long)c3[3 * j + 1] - c3[3 * i + 1];
    long long dz = (long long)c3[3 * j + 2] - c3[3 * i + 2];
    long long a = nint[3 * i] * dx + nint[3 * i + 1] * dy + nint[3 * i + 2] * dz;
    long long b = nint[3 * j] * dx + nint[3 * j + 1] * dy + nint[3 * j + 2] * dz;
    return a > 0 && b < 0;
}

__device__ __forceinline__ bool pair_visible(const int32_t* __restrict__ c3, const long long* __restrict__ nint,
                                             const BvhNode* __restrict__ nodes, const BvhTri* __restrict__ tris,
                                             int fi, int fj) {
    if (fi == fj || !cull_pass(c3, nint, fi, fj)) return false;
    int a = fi < fj ? fi : fj, b = fi < fj ? fj : fi;
    P3 P{c3[3 * a], c3[3 * a + 1], c3[3 * a + 2]};
    P3 Q{c3[3 * b], c3[3 * b + 1], c3[3 * b + 2]};
    return !bvh_blocked<0>(nodes, tris, P, Q, a, b);
}

// ------------------------------------------------------------ kernels
__global__ void k_minmax(const double* __restrict__ v, int64_t nv, double* out) {
    __shared__ double slo[3][256], shi[3][256];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = threadIdx.x; i < nv; i += blockDim.x)
        for (int a = 0; a < 3; ++a) {
            double x = v[3 * i + a];
            lo[a] = fmin(lo[a], x);
            hi[a] = fmax(hi[a], x);
        }
    for (int a = 0; a < 3; ++a) { slo[a][threadIdx.x] = lo[a]; shi[a][threadIdx.x] = hi[a]; }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int a = 0; a < 3; ++a) {
                slo[a][threadIdx.x] = fmin(slo[a][threadIdx.x], slo[a][threadIdx.x + s]);
                shi[a][threadIdx.x] = fmax(shi[a][threadIdx.x], shi[a][threadIdx.x + s]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int a = 0; a < 3; ++a) { out[a] = slo[a][0]; out[3 + a] = shi[a][0]; }
}

__global__ void k_snap(const double* __restrict__ v, int64_t nv, double unit, long long b0, long long b1,
                       long long b2, int32_t* __restrict__ q) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nv) return;
    q[3 * i + 0] = (int32_t)(llround(v[3 * i + 0] / unit) - b0);
    q[3 * i + 1] = (int32_t)(llround(v[3 * i + 1] / unit) - b1);
    q[3 * i + 2] = (int32_t)(llround(v[3 * i + 2] / unit) - b2);
}

__global__ void k_geometry(const int32_t* __restrict__ q, const int32_t* __restrict__ f, int64_t nf, double unit,
                           int32_t* __restrict__ c3, long long* __restrict__ nint, double* __restrict__ area,
                           double* __restrict__ cent, double* __restrict__ nrm) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nf) return;
    const int32_t* A = q + 3 * (int64_t)f[3 * t];
    const int32_t* B = q + 3 * (int64_t)f[3 * t + 1];
    const int32_t* C = q + 3 * (int64_t)f[3 * t + 2];
    long long ux = B[0] - A[0], uy = B[1] - A[1], uz = B[2] - A[2];
    long long wx = C[0] - A[0], wy = C[1] - A[1], wz = C[2] - A[2];
    nint[3 * t + 0] = uy * wz - uz * wy;
    nint[3 * t + 1] = uz * wx - ux * wz;
    nint[3 * t + 2] = ux * wy - uy * wx;
    for (int a = 0; a < 3; ++a) c3[3 * t + a] = A[a] + B[a] + C[a];
    double a0 = A[0] * unit, a1 = A[1] * unit, a2 = A[2] * unit;
    double b0 = B[0] * unit, b1 = B[1] * unit, b2 = B[2] * unit;
    double d0 = C[0] * unit, d1 = C[1] * unit, d2 = C[2] * unit;
    double u0 = b0 - a0, u1 = b1 - a1, u2 = b2 - a2;
    double w0 = d0 - a0, w1 = d1 - a1, w2 = d2 - a2;
    double n0 = u1 * w2 - u2 * w1, n1 = u2 * w0 - u0 * w2, n2 = u0 * w1 - u1 * w0;
    double len = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
    area[t] = 0.5 * len;
    cent[3 * t + 0] = (a0 + b0 + d0) / 3.0;
    cent[3 * t + 1] = (a1 + b1 + d1) / 3.0;
    cent[3 * t + 2] = (a2 + b2 + d2) / 3.0;
    double inv = len > 0 ? 1.0 / len : 0.0;
    nrm[3 * t + 0] = n0 * inv;
    nrm[3 * t + 1] = n1 * inv;
    nrm[3 * t + 2] = n2 * inv;
}

// V rows (facet order) for vf_mesh_visibility: one thread per (row, j).
__global__ void k_vis_rows(const int32_t* __restrict__ c3, const long long* __restrict__ nint,
                           const BvhNode* __restrict__ nodes, const BvhTri* __restrict__ tris, int64_t nf,
                           const int64_t* __restrict__ rows, int64_t nrows, uint8_t* __restrict__ V) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nrows * nf) return;
    int64_t r = idx / nf;
    int j = (int)(idx - r * nf);
    int i = (int)rows[r];
    V[idx] = pair_visible(c3, nint, nodes, tris, i, j) ? 1 : 0;
}

// Upper-triangle words of the bit matrix in index order: one CTA per row i,
// one warp per 32-column word (ballot over lanes); words left of the
// diagonal are written 0 and filled by the transpose kernel.
__global__ void k_vis_bits_upper(const int32_t* __restrict__ c3, const long long* __restrict__ nint,
                                 const BvhNode* __restrict__ nodes, const BvhTri* __restrict__ tris,
                                 const int32_t* __restrict__ index, int64_t n, int64_t row0,
                                 uint32_t* __restrict__ bits, int64_t ldw) {
    int64_t i = row0 + blockIdx.x;
    if (i >= n) return;
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    int fi = index[i];
    int64_t wdiag = i >> 5;
    uint32_t* row = bits + i * ldw;
    for (int64_t w = warp; w < wdiag; w += nw)
        if (lane == 0) row[w] = 0u;
    for (int64_t w = wdiag + warp; w < ldw; w += nw) {
        int64_t j = (w << 5) + lane;
        bool v = false;
        if (j > i && j < n) v = pair_visible(c3, nint, nodes, tris, fi, index[j]);
        uint32_t word = __ballot_sync(0xffffffffu, v);
        if (lane == 0) row[w] = word;
    }
}

// Mirror the upper triangle into the lower one: for a 32x32 tile (I, W),
// W >= I, lane r holds row 32I+r's word W; bit c of the transposed tile row
// c is that lane-ballot.  Diagonal tiles OR the two halves.
__global__ void k_vis_bits_mirror(uint32_t* __restrict__ bits, int64_t n, int64_t ldw, int64_t ntile_rows) {
    int64_t warp_global = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    // enumerate tiles (I, W) with W >= I row by row
    int64_t I = 0, acc = 0;
    // find I such that acc(I) <= warp_global < acc(I+1); rows have (ntile_rows - I) tiles
    // closed form via the triangular count would be faster; a binary search keeps it exact
    int64_t lo = 0, hi = ntile_rows;
    auto start = [&](int64_t r) { return r * ntile_rows - r * (r - 1) / 2; };
    int64_t total = start(ntile_rows);
    if (warp_global >= total) return;
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) / 2;
        if (start(mid) <= warp_global) lo = mid; else hi = mid;
    }
    I = lo;
    acc = start(I);
    int64_t W = I + (warp_global - acc);
    int64_t r = 32 * I + lane;
    uint32_t u = (r < n) ? bits[r * ldw + W] : 0u;
    uint32_t t = 0;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        uint32_t col = __ballot_sync(0xffffffffu, (u >> c) & 1u);
        if (lane == c) t = col;
    }
    int64_t rr = 32 * W + lane;
    if (W == I) {
        if (r < n) bits[r * ldw + W] = u | t;
    } else if (rr < n) {
        bits[rr * ldw + I] = t;
    }
}

__global__ void k_insolation(const int32_t* __restrict__ c3, const long long* __restrict__ nint,
                             const double* __restrict__ nrm, const BvhNode* __restrict__ nodes,
                             const BvhTri* __restrict__ tris, int64_t nf, const double* __restrict__ dirs,
                             const long long* __restrict__ dq, int R, double S, float* __restrict__ E,
                             int64_t lde) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nf * (int64_t)R) return;
    int r = (int)(idx / nf);
    int i = (int)(idx - (int64_t)r * nf);
    P3 D{dq[3 * r], dq[3 * r + 1], dq[3 * r + 2]};
    long long nd = nint[3 * i] * D.x + nint[3 * i + 1] * D.y + nint[3 * i + 2] * D.z;
    float e = 0.f;
    if (nd > 0) {
        P3 P{c3[3 * i], c3[3 * i + 1], c3[3 * i + 2]};
        if (!bvh_blocked<1>(nodes, tris, P, D, i, -1)) {
            double c = nrm[3 * i] * dirs[3 * r] + nrm[3 * i + 1] * dirs[3 * r + 1] + nrm[3 * i + 2] * dirs[3 * r + 2];
            e = (float)(S * fmax(0.0, c));
        }
    }
    E[i + (int64_t)r * lde] = e;
}

// Finite solar disk (Section 2: a sum over point sources): per (facet,
// sun) the weighted sum of the point-sun insolation of the disk's M sample
// directions dirs[r * M + k] with weights w[k], summed in FP64 in k order.
__global__ void k_insolation_disk(const int32_t* __restrict__ c3, const long long* __restrict__ nint,
                                  const double* __restrict__ nrm, const BvhNode* __restrict__ nodes,
                                  const BvhTri* __restrict__ tris, int64_t nf, const double* __restrict__ dirs,
                                  const long long* __restrict__ dq, const double* __restrict__ w, int M, int R,
                                  double S, float* __restrict__ E, int64_t lde) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nf * (int64_t)R) return;
    const int r = (int)(idx / nf);
    const int i = (int)(idx - (int64_t)r * nf);
    const P3 P{c3[3 * i], c3[3 * i + 1], c3[3 * i + 2]};
    double e = 0.0;
    for (int k = 0; k < M; ++k) {
        const int64_t d = (int64_t)r * M + k;
        const P3 D{dq[3 * d], dq[3 * d + 1], dq[3 * d + 2]};
        const long long nd = nint[3 * i] * D.x + nint[3 * i + 1] * D.y + nint[3 * i + 2] * D.z;
        if (nd <= 0 || bvh_blocked<1>(nodes, tris, P, D, i, -1)) continue;
        const double c = nrm[3 * i] * dirs[3 * d] + nrm[3 * i + 1] * dirs[3 * d + 1] + nrm[3 * i + 2] * dirs[3 * d + 2];
        e += w[k] * S * fmax(0.0, c);
    }
    E[i + (int64_t)r * lde] = (float)e;
}

// The disk's sample directions around the unit direction s: rings of equal
// radial width (ring k split into max(1, 6k) equal sectors), each cell's
// point at its area-weighted mean radius and mid angle, weight = its share
// of the disk's area.
static void disk_samples(const double* s_in, double radius, int rings, std::vector<double>& dirs,
                         std::vector<double>& wts) {
    double s[3] = {s_in[0], s_in[1], s_in[2]};
    const double sn = std::sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    for (double& x : s) x /= sn;
    const double a[3] = {std::fabs(s[0]) < 0.9 ? 1.0 : 0.0, std::fabs(s[0]) < 0.9 ? 0.0 : 1.0, 0.0};
    double u[3] = {s[1] * a[2] - s[2] * a[1], s[2] * a[0] - s[0] * a[2], s[0] * a[1] - s[1] * a[0]};
    const double un = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (double& x : u) x /= un;
    const double v[3] = {s[1] * u[2] - s[2] * u[1], s[2] * u[0] - s[0] * u[2], s[0] * u[1] - s[1] * u[0]};
    wts.clear();
    for (int k = 0; k < rings; ++k) {
        const double r0 = (double)k / rings, r1 = (double)(k + 1) / rings;
        const int nsec = k == 0 ? 1 : 6 * k;
        const double share = (r1 * r1 - r0 * r0) / nsec;
        const double rc = k == 0 ? 0.0 : (2.0 / 3.0) * (r1 * r1 * r1 - r0 * r0 * r0) / (r1 * r1 - r0 * r0);
        const double t = radius * rc;
        for (int j = 0; j < nsec; ++j) {
            const double phi = 2.0 * M_PI * (j + 0.5) / nsec;
            double d[3];
            for (int c = 0; c < 3; ++c)
                d[c] = std::cos(t) * s[c] + std::sin(t) * (std::cos(phi) * u[c] + std::sin(phi) * v[c]);
            const double dn = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            for (int c = 0; c < 3; ++c) dirs.push_back(d[c] / dn);
            wts.push_back(share);
        }
    }
}

// ------------------------------------------------------------ BVH build
// Median split on the longest axis of the centroid bounds, leaves <= 4
// triangles; children allocated in adjacent slots.  Host code: integer
// work on N centroids, O(N log^2 N).
vf_status bvh_build(vf_mesh* m) {
    const int64_t nf = m->nf;
    std::vector<int32_t> hq;
    VF_TRY(m->q.download(hq));
    std::vector<int32_t> order(nf);
    for (int64_t i = 0; i < nf; ++i) order[i] = (int32_t)i;
    const std::vector<int32_t>& c3 = m->h_c3;
    std::vector<BvhNode> nodes;
    nodes.reserve(2 * nf / 4 + 8);
    struct Item { int32_t node, first, count, depth; };
    std::vector<Item> st;
    nodes.push_back(BvhNode{});
    st.push_back({0, 0, (int32_t)nf, 1});
    int maxdepth = 1;
    auto tri_box = [&](int32_t f, int32_t lo[3], int32_t hi[3]) {
        for (int v = 0; v < 3; ++v) {
            int32_t vi = m->h_faces[3 * (int64_t)f + v];
            for (int a = 0; a < 3; ++a) {
                int32_t x = 3 * hq[3 * (int64_t)vi + a];
                lo[a] = std::min(lo[a], x);
                hi[a] = std::max(hi[a], x);
            }
        }
    };
    while (!st.empty()) {
        Item it = st.back();
        st.pop_back();
        maxdepth = std::max(maxdepth, it.depth);
        BvhNode nd;
        int32_t clo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, chi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
        for (int a = 0; a < 3; ++a) { nd.lo[a] = INT32_MAX; nd.hi[a] = INT32_MIN; }
        for (int32_t s = it.first; s < it.first + it.count; ++s) {
            int32_t f = order[s];
            tri_box(f, nd.lo, nd.hi);
            for (int a = 0; a < 3; ++a) {
                clo[a] = std::min(clo[a], c3[3 * (int64_t)f + a]);
                chi[a] = std::max(chi[a], c3[3 * (int64_t)f + a]);
            }
        }
        if (it.count <= 4) {
            nd.left = it.first;
            nd.count = it.count;
            nodes[it.node] = nd;
            continue;
        }
        int ax = 0;
        for (int a = 1; a < 3; ++a)
            if (chi[a] - clo[a] > chi[ax] - clo[ax]) ax = a;
        int32_t half = it.count / 2;
        std::nth_element(order.begin() + it.first, order.begin() + it.first + half,
                         order.begin() + it.first + it.count, [&](int32_t x, int32_t y) {
                             int32_t kx = c3[3 * (int64_t)x + ax], ky = c3[3 * (int64_t)y + ax];
                             return kx != ky ? kx < ky : x < y;
                         });
        int32_t l = (int32_t)nodes.size();
        nodes.push_back(BvhNode{});
        nodes.push_back(BvhNode{});
        nd.left = l;
        nd.count = 0;
        nodes[it.node] = nd;
        st.push_back({l + 1, it.first + half, it.count - half, it.depth + 1});
        st.push_back({l, it.first, half, it.depth + 1});
    }
    VF_CHECK(maxdepth + 2 < kStack, VF_E_INVAL, "BVH depth %d exceeds the traversal stack", maxdepth);
    std::vector<BvhTri> tris(nf);
    for (int64_t s = 0; s < nf; ++s) {
        int32_t f = order[s];
        BvhTri t{};
        for (int v = 0; v < 3; ++v) {
            int32_t vi = m->h_faces[3 * (int64_t)f + v];
            for (int a = 0; a < 3; ++a) t.v[3 * v + a] = 3 * hq[3 * (int64_t)vi + a];
        }
        t.facet = f;
        tris[s] = t;
    }
    VF_TRY(m->bvh_nodes.upload(nodes));
    VF_TRY(m->bvh_tris.upload(tris));
    m->bvh_depth = maxdepth;
    return VF_OK;
}

vf_status visibility_bits(const vf_mesh* m, const int32_t* d_index, int64_t n, uint32_t* d_bits, int64_t ldw,
                          cudaStream_t st) {
    const int64_t chunk = 1 << 16;  // rows per launch (grid.x limit is large; chunking bounds each launch)
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        int64_t rows = std::min(chunk, n - r0);
        k_vis_bits_upper<<<(unsigned)rows, 256, 0, st>>>(m->c3.p, m->nint.p, m->bvh_nodes.p, m->bvh_tris.p,
                                                         d_index, n, r0, d_bits, ldw);
        VF_TRY_CUDA(cudaGetLastError());
    }
    int64_t ntr = ceil_div(n, 32);
    int64_t tiles = ntr * (ntr + 1) / 2;
    int64_t threads = tiles * 32;
    k_vis_bits_mirror<<<(unsigned)ceil_div(threads, 256), 256, 0, st>>>(d_bits, n, ldw, ntr);
    VF_TRY_CUDA(cudaGetLastError());
    return VF_OK;
}

}  // namespace vf

using namespace vf;

// ============================================================ C ABI
extern "C" const char* vf_last_error(void) { return vf::g_err; }
extern "C" const char* vf_version(void) { return "libvf 0.2 (sm_103a)"; }

extern "C" vf_status vf_debug_fail_alloc(int64_t nth) {
    clear_error();
    VF_CHECK(nth >= 0, VF_E_INVAL, "vf_debug_fail_alloc: nth must be >= 0");
    g_fail_alloc.store(nth, std::memory_order_relaxed);
    return VF_OK;
}

extern "C" vf_status vf_mesh_create(const double* verts, int64_t nv, const int32_t* faces, int64_t nf,
                                    const vf_mesh_opts* opts, vf_mesh** out) {
    clear_error();
    VF_CHECK(out && verts && faces, VF_E_INVAL, "vf_mesh_create: null pointer");
    *out = nullptr;
    VF_CHECK(nv >= 3 && nf >= 1, VF_E_INVAL, "vf_mesh_create: need nv >= 3 and nf >= 1 (got %lld, %lld)",
             (long long)nv, (long long)nf);
    VF_CHECK(nf < (1ll << 31) && nv < (1ll << 31), VF_E_INVAL, "vf_mesh_create: mesh too large");
    for (int64_t i = 0; i < 3 * nf; ++i)
        VF_CHECK(faces[i] >= 0 && faces[i] < nv, VF_E_INVAL, "vf_mesh_create: face index %d out of range",
                 faces[i]);
    int dev = opts ? opts->device : 0;
    device_guard g(dev);
    VF_TRY_CUDA(cudaSetDevice(dev));
    vf_mesh* m = new vf_mesh();
    m->device = dev;
    m->nf = nf;
    m->nv = nv;
    m->h_faces.assign(faces, faces + 3 * nf);
    auto fail = [&](vf_status s) { delete m; return s; };
    dbuf<double> dv, mm;
    vf_status s;
    if ((s = dv.upload(verts, 3 * nv)) != VF_OK) return fail(s);
    if ((s = mm.alloc(6)) != VF_OK) return fail(s);
    k_minmax<<<1, 256>>>(dv.p, nv, mm.p);
    double hmm[6];
    if (cudaMemcpy(hmm, mm.p, sizeof(hmm), cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("vf_mesh_create: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(VF_E_CUDA);
    }
    double ext = 0;
    for (int a = 0; a < 3; ++a) ext = std::max(ext, hmm[3 + a] - hmm[a]);
    if (!(ext > 0) || !std::isfinite(ext)) {
        set_error("vf_mesh_create: vertex set has zero or non-finite extent");
        return fail(VF_E_INVAL);
    }
    int ex;
    std::frexp(ext, &ex);
    m->unit = std::ldexp(1.0, ex - 18);
    for (int a = 0; a < 3; ++a) m->base[a] = std::llround(hmm[a] / m->unit);
    if ((s = m->q.alloc(3 * nv)) != VF_OK) return fail(s);
    k_snap<<<(unsigned)ceil_div(nv, 256), 256>>>(dv.p, nv, m->unit, m->base[0], m->base[1], m->base[2], m->q.p);
    if ((s = m->faces.upload(faces, 3 * nf)) != VF_OK) return fail(s);
    if ((s = m->c3.alloc(3 * nf)) != VF_OK || (s = m->nint.alloc(3 * nf)) != VF_OK ||
        (s = m->area.alloc(nf)) != VF_OK || (s = m->cent.alloc(3 * nf)) != VF_OK ||
        (s = m->nrm.alloc(3 * nf)) != VF_OK)
        return fail(s);
    k_geometry<<<(unsigned)ceil_div(nf, 256), 256>>>(m->q.p, m->faces.p, nf, m->unit, m->c3.p, m->nint.p, m->area.p,
                                                     m->cent.p, m->nrm.p);
    if ((s = m->c3.download(m->h_c3)) != VF_OK) return fail(s);
    if (cudaGetLastError() != cudaSuccess) {
        set_error("vf_mesh_create: geometry kernel failed");
        return fail(VF_E_CUDA);
    }
    if ((s = bvh_build(m)) != VF_OK) return fail(s);
    *out = m;
    return VF_OK;
}

extern "C" void vf_mesh_destroy(vf_mesh* m) {
    if (!m) return;
    device_guard g(m->device);
    delete m;
}

extern "C" int64_t vf_mesh_nfacets(const vf_mesh* m) { return m ? m->nf : -1; }

extern "C" vf_status vf_mesh_grid(const vf_mesh* m, double* unit, int64_t base[3]) {
    clear_error();
    VF_CHECK(m, VF_E_INVAL, "vf_mesh_grid: null mesh");
    if (unit) *unit = m->unit;
    if (base)
        for (int a = 0; a < 3; ++a) base[a] = m->base[a];
    return VF_OK;
}

extern "C" vf_status vf_mesh_geometry(const vf_mesh* m, double* area, double* centroid, double* normal) {
    clear_error();
    VF_CHECK(m, VF_E_INVAL, "vf_mesh_geometry: null mesh");
    device_guard g(m->device);
    if (area) VF_TRY_CUDA(cudaMemcpy(area, m->area.p, m->nf * sizeof(double), cudaMemcpyDeviceToHost));
    if (centroid) VF_TRY_CUDA(cudaMemcpy(centroid, m->cent.p, 3 * m->nf * sizeof(double), cudaMemcpyDeviceToHost));
    if (normal) VF_TRY_CUDA(cudaMemcpy(normal, m->nrm.p, 3 * m->nf * sizeof(double), cudaMemcpyDeviceToHost));
    return VF_OK;
}

extern "C" vf_status vf_mesh_visibility(const vf_mesh* m, const int64_t* rows, int64_t nrows, uint8_t* V) {
    clear_error();
    VF_CHECK(m && V, VF_E_INVAL, "vf_mesh_visibility: null argument");
    if (!rows) nrows = m->nf;
    VF_CHECK(nrows >= 0, VF_E_INVAL, "vf_mesh_visibility: nrows < 0");
    if (rows)
        for (int64_t r = 0; r < nrows; ++r)
            VF_CHECK(rows[r] >= 0 && rows[r] < m->nf, VF_E_INVAL, "vf_mesh_visibility: row %lld out of range",
                     (long long)rows[r]);
    if (nrows == 0) return VF_OK;
    device_guard g(m->device);
    const int64_t chunk_rows = std::max<int64_t>(1, (int64_t(1) << 28) / m->nf);
    dbuf<uint8_t> dV;
    dbuf<int64_t> drows;
    VF_TRY(dV.alloc(std::min(chunk_rows, nrows) * m->nf));
    VF_TRY(drows.alloc(std::min(chunk_rows, nrows)));
    std::vector<int64_t> idx;
    for (int64_t r0 = 0; r0 < nrows; r0 += chunk_rows) {
        int64_t nr = std::min(chunk_rows, nrows - r0);
        idx.resize(nr);
        for (int64_t k = 0; k < nr; ++k) idx[k] = rows ? rows[r0 + k] : r0 + k;
        VF_TRY_CUDA(cudaMemcpy(drows.p, idx.data(), nr * sizeof(int64_t), cudaMemcpyHostToDevice));
        int64_t tot = nr * m->nf;
        k_vis_rows<<<(unsigned)ceil_div(tot, 256), 256>>>(m->c3.p, m->nint.p, m->bvh_nodes.p, m->bvh_tris.p, m->nf,
                                                          drows.p, nr, dV.p);
        VF_TRY_CUDA(cudaGetLastError());
        VF_TRY_CUDA(cudaMemcpy(V + r0 * m->nf, dV.p, tot, cudaMemcpyDeviceToHost));
    }
    return VF_OK;
}

extern "C" vf_status vf_mesh_insolation(const vf_mesh* m, const double* sun_dirs, int32_t R, double solar_flux,
                                        float* E, int64_t lde, vf_stream stream) {
    clear_error();
    VF_CHECK(m && sun_dirs && E, VF_E_INVAL, "vf_mesh_insolation: null argument");
    VF_CHECK(R >= 1 && lde >= m->nf, VF_E_INVAL, "vf_mesh_insolation: need R >= 1 and lde >= nf");
    device_guard g(m->device);
    std::vector<long long> dq(3 * (size_t)R);
    for (int64_t k = 0; k < 3 * (int64_t)R; ++k) dq[k] = std::llround(std::ldexp(sun_dirs[k], 20));
    dbuf<double> ddirs;
    dbuf<long long> ddq;
    VF_TRY(ddirs.upload(sun_dirs, 3 * (size_t)R));
    VF_TRY(ddq.upload(dq));
    int64_t tot = m->nf * (int64_t)R;
    k_insolation<<<(unsigned)ceil_div(tot, 256), 256, 0, (cudaStream_t)stream>>>(
        m->c3.p, m->nint.p, m->nrm.p, m->bvh_nodes.p, m->bvh_tris.p, m->nf, ddirs.p, ddq.p, R, solar_flux, E, lde);
    VF_TRY_CUDA(cudaGetLastError());
    // the staging buffers are freed on return: order that after the kernel
    VF_TRY_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return VF_OK;
}

extern "C" vf_status vf_mesh_insolation_disk(const vf_mesh* m, const double* sun_dirs, int32_t R, double solar_flux,
                                             double angular_radius, int32_t rings, float* E, int64_t lde,
                                             vf_stream stream) {
    clear_error();
    VF_CHECK(m && sun_dirs && E, VF_E_INVAL, "vf_mesh_insolation_disk: null argument");
    VF_CHECK(R >= 1 && lde >= m->nf, VF_E_INVAL, "vf_mesh_insolation_disk: need R >= 1 and lde >= nf");
    VF_CHECK(rings >= 1 && rings <= 64 && angular_radius >= 0 && angular_radius < 0.5, VF_E_INVAL,
             "vf_mesh_insolation_disk: need 1 <= rings <= 64 and 0 <= angular_radius < 0.5 rad");
    device_guard g(m->device);
    std::vector<double> dirs, w;
    for (int32_t r = 0; r < R; ++r) disk_samples(sun_dirs + 3 * (size_t)r, angular_radius, rings, dirs, w);
    const int M = (int)w.size();  // the same weights for every sun (disk_samples refills them per sun)
    VF_CHECK((int64_t)dirs.size() == 3 * (int64_t)M * R, VF_E_INVAL, "vf_mesh_insolation_disk: sample count");
    std::vector<long long> dq(dirs.size());
    for (size_t k = 0; k < dirs.size(); ++k) dq[k] = std::llround(std::ldexp(dirs[k], 20));
    dbuf<double> ddirs, dw;
    dbuf<long long> ddq;
    VF_TRY(ddirs.upload(dirs));
    VF_TRY(ddq.upload(dq));
    VF_TRY(dw.upload(w));
    const int64_t tot = m->nf * (int64_t)R;
    k_insolation_disk<<<(unsigned)ceil_div(tot, 128), 128, 0, (cudaStream_t)stream>>>(
        m->c3.p, m->nint.p, m->nrm.p, m->bvh_nodes.p, m->bvh_tris.p, m->nf, ddirs.p, ddq.p, dw.p, M, R, solar_flux,
        E, lde);
    VF_TRY_CUDA(cudaGetLastError());
    VF_TRY_CUDA(cudaStreamSynchronize((cudaStream_t)stream));  // the staging buffers are freed on return
    return VF_OK;
}

// ============================================================ partition
extern "C" vf_status vf_partition(const vf_mesh* m, const vf_partition_opts* opts, vf_tree** out) {
    clear_error();
    VF_CHECK(m && out, VF_E_INVAL, "vf_partition: null argument");
    *out = nullptr;
    int kind = opts ? opts->kind : VF_TREE_QUAD;
    int leaf = opts && opts->leaf_size > 0 ? opts->leaf_size : 64;
    int maxd = opts && opts->max_depth > 0 ? opts->max_depth : 32;
    VF_CHECK(kind == VF_TREE_QUAD || kind == VF_TREE_OCT, VF_E_INVAL, "vf_partition: bad tree kind %d", kind);
    const int axes = kind == VF_TREE_QUAD ? 2 : 3;
    const int nch = 1 << axes;
    const int64_t n = m->nf;
    vf_tree* t = new vf_tree();
    t->kind = kind;
    t->leaf_size = leaf;
    t->max_depth = maxd;
    t->nf = n;
    std::vector<int32_t> work(n), tmp(n);
    for (int64_t i = 0; i < n; ++i) work[i] = (int32_t)i;
    const std::vector<int32_t>& c3 = m->h_c3;
    // preorder DFS: each stack item is a range of `work` plus its parent id
    struct Item { int32_t first, count, depth, parent; };
    std::vector<Item> st;
    st.push_back({0, (int32_t)n, 0, -1});
    while (!st.empty()) {
        Item it = st.back();
        st.pop_back();
        int32_t id = (int32_t)t->first.size();
        t->first.push_back(it.first);
        t->count.push_back(it.count);
        t->depth.push_back(it.depth);
        t->parent.push_back(it.parent);
        t->kids.emplace_back();
        if (it.parent >= 0) t->kids[it.parent].push_back(id);
        if (it.count <= leaf || it.depth >= maxd) continue;
        int32_t lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
        for (int32_t s = it.first; s < it.first + it.count; ++s)
            for (int a = 0; a < axes; ++a) {
                int32_t x = c3[3 * (int64_t)work[s] + a];
                lo[a] = std::min(lo[a], x);
                hi[a] = std::max(hi[a], x);
            }
        bool flat = true;
        for (int a = 0; a < axes; ++a) flat = flat && lo[a] == hi[a];
        if (flat) continue;
        // stable counting sort of the range by child code
        int32_t cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        auto code_of = [&](int32_t f) {
            int c = 0;
            for (int a = 0; a < axes; ++a)
                c = 2 * c + (2 * (int64_t)c3[3 * (int64_t)f + a] >= (int64_t)lo[a] + hi[a] ? 1 : 0);
            return c;
        };
        for (int32_t s = it.first; s < it.first + it.count; ++s) cnt[code_of(work[s])]++;
        int32_t off[8];
        int32_t acc = it.first;
        for (int c = 0; c < nch; ++c) { off[c] = acc; acc += cnt[c]; }
        int32_t pos[8];
        for (int c = 0; c < nch; ++c) pos[c] = off[c];
        for (int32_t s = it.first; s < it.first + it.count; ++s) tmp[pos[code_of(work[s])]++] = work[s];
        std::copy(tmp.begin() + it.first, tmp.begin() + it.first + it.count, work.begin() + it.first);
        for (int c = nch - 1; c >= 0; --c)
            if (cnt[c] > 0) st.push_back({off[c], cnt[c], it.depth + 1, id});
    }
    t->perm = std::move(work);
    *out = t;
    return VF_OK;
}

extern "C" void vf_tree_destroy(vf_tree* t) { delete t; }
extern "C" int64_t vf_tree_nnodes(const vf_tree* t) { return t ? (int64_t)t->first.size() : -1; }

extern "C" vf_status vf_tree_perm(const vf_tree* t, int32_t* perm) {
    clear_error();
    VF_CHECK(t && perm, VF_E_INVAL, "vf_tree_perm: null argument");
    std::copy(t->perm.begin(), t->perm.end(), perm);
    return VF_OK;
}

extern "C" vf_status vf_tree_nodes(const vf_tree* t, int32_t* first, int32_t* count, int32_t* depth,
                                   int32_t* parent) {
    clear_error();
    VF_CHECK(t, VF_E_INVAL, "vf_tree_nodes: null tree");
    if (first) std::copy(t->first.begin(), t->first.end(), first);
    if (count) std::copy(t->count.begin(), t->count.end(), count);
    if (depth) std::copy(t->depth.begin(), t->depth.end(), depth);
    if (parent) std::copy(t->parent.begin(), t->parent.end(), parent);
    return VF_OK;
}
