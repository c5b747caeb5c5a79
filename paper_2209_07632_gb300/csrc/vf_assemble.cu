// Assembly of the compressed view-factor matrix (Algorithms 1, 3, 4).
//
// Device side: tree-order geometry, the pair-visibility bit matrix, per
// leaf-pair statistics, matrix-free block SVD probes (randomized subspace
// iteration + one-sided Jacobi) and payload packing.  Host side: the
// dynamic programme of Algorithm 4 over block pairs, processed bottom-up by
// block height so each level's probes run as one batch of launches.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <numeric>

#include "vf_hmat.cuh"
#include "vf_predictor.cuh"

namespace vf {

constexpr float kPi = 3.14159265358979323846f;
constexpr int kMaxEll = 160;   // largest probe subspace (shared-memory Jacobi)
// Rank-predictor audits: one in kAuditEvery predicted skips is probed
// anyway; if more than one in kAuditMaxWinInv of a level's audits (and at
// least two) would have stored an SVD, that level's skips are probed too.
constexpr int64_t kAuditEvery = 8;
constexpr int64_t kAuditMaxWinInv = 4;

// ------------------------------------------------------------ geometry
struct Geo {
    const float4* xa;     // scale-3 integer centroid as floats, area
    const float4* nv;     // unit normal
    const uint32_t* bits; // visibility, tree order
    int64_t ldw;
    float s;              // grid unit / 3
};

__global__ void k_tree_geom(const int32_t* __restrict__ perm, const int32_t* __restrict__ c3,
                            const double* __restrict__ area, const double* __restrict__ nrm, int64_t n,
                            float4* __restrict__ xa, float4* __restrict__ nv) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    int64_t f = perm[t];
    xa[t] = make_float4((float)c3[3 * f], (float)c3[3 * f + 1], (float)c3[3 * f + 2], (float)area[f]);
    nv[t] = make_float4((float)nrm[3 * f], (float)nrm[3 * f + 1], (float)nrm[3 * f + 2], 0.f);
}

// F_ij (Eq. FF-def) in tree order; the coordinate difference is exact
// (integers < 2^21) before the single scaling by unit/3.
__device__ __forceinline__ float entry(const Geo& g, int i, int j) {
    uint32_t w = __ldg(g.bits + (int64_t)i * g.ldw + (j >> 5));
    if (!((w >> (j & 31)) & 1u)) return 0.f;
    float4 a = __ldg(g.xa + i), b = __ldg(g.xa + j);
    float4 na = __ldg(g.nv + i), nb = __ldg(g.nv + j);
    float dx = (b.x - a.x) * g.s, dy = (b.y - a.y) * g.s, dz = (b.z - a.z) * g.s;
    float r2 = dx * dx + dy * dy + dz * dz;
    float ci = na.x * dx + na.y * dy + na.z * dz;
    float cj = -(nb.x * dx + nb.y * dy + nb.z * dz);
    return ci * cj * b.w / (kPi * r2 * r2);
}

// ------------------------------------------------------------ leaf pairs
// One warp per (row leaf a, column leaf b); leaves hold <= 64 facets.  For
// each row r of leaf a, the 64-bit window of its visibility bits over leaf
// b's columns gives the row's nonzeros.
__global__ void k_leaf_pair_stats(const uint32_t* __restrict__ bits, int64_t ldw, const int32_t* __restrict__ lf,
                                  const int32_t* __restrict__ lc, int64_t nleaves, int64_t p0, int64_t np,
                                  unsigned long long* __restrict__ rowmask, unsigned long long* __restrict__ colmask,
                                  int32_t* __restrict__ nnz) {
    int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (wid >= np) return;
    int64_t p = p0 + wid;
    int64_t a = p / nleaves, b = p - a * nleaves;
    int r0 = lf[a], m = lc[a], c0 = lf[b], n = lc[b];
    int64_t w0 = c0 >> 5;
    int sh = c0 & 31;
    unsigned long long cmask = 0;
    int cnt = 0;
    unsigned long long nmask = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
    uint32_t rb[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        int r = lane + 32 * h;
        unsigned long long win = 0;
        if (r < m) {
            const uint32_t* row = bits + (int64_t)(r0 + r) * ldw;
            unsigned long long lo = row[w0];
            if (w0 + 1 < ldw) lo |= (unsigned long long)row[w0 + 1] << 32;
            unsigned long long hi = (w0 + 2 < ldw) ? row[w0 + 2] : 0ull;
            win = sh ? ((lo >> sh) | (hi << (64 - sh))) : lo;
            win &= nmask;
        }
        cmask |= win;
        cnt += __popcll(win);
        rb[h] = __ballot_sync(0xffffffffu, win != 0ull);
    }
    unsigned int clo = __reduce_or_sync(0xffffffffu, (unsigned int)(cmask & 0xffffffffu));
    unsigned int chi = __reduce_or_sync(0xffffffffu, (unsigned int)(cmask >> 32));
    int tot = __reduce_add_sync(0xffffffffu, cnt);
    if (lane == 0) {
        rowmask[wid] = (unsigned long long)rb[0] | ((unsigned long long)rb[1] << 32);
        colmask[wid] = (unsigned long long)clo | ((unsigned long long)chi << 32);
        nnz[wid] = tot;
    }
}

// ------------------------------------------------------------ probes
struct ProbeDesc {
    int64_t rows_off, cols_off; // into the index list (tree positions)
    int32_t m1, n1, ell, pad;
    int64_t y_off;              // m1 x ell panel (column-major)
    int64_t z_off;              // n1 x ell panel
    int64_t s_off;              // ell x ell small matrices (M then W), and ell sigmas
    uint64_t seed;
};

struct PanelItem {
    int32_t probe;
    int32_t o0;  // first output row
    int32_t c0;  // first panel column
    int32_t pad;
};

// Out = A * In (TRANS = false: out rows are A's rows, contraction over its
// columns) or Out = A^T * In (TRANS = true).  A is evaluated on the fly.
// RANDOM: In is a seeded uniform(-1,1) panel instead of memory.  Tile: 32 output
// rows x 32 panel columns, 128 threads, 8 outputs per thread.
template <bool TRANS, bool RANDOM>
__global__ void __launch_bounds__(128) k_apanel(Geo g, const ProbeDesc* __restrict__ pd,
                                                const PanelItem* __restrict__ items, const int32_t* __restrict__ idx,
                                                const float* __restrict__ pin, float* __restrict__ pout) {
    __shared__ float As[32][33];
    __shared__ float Ps[32][33];
    const PanelItem it = items[blockIdx.x];
    const ProbeDesc d = pd[it.probe];
    const int out_n = TRANS ? d.n1 : d.m1;
    const int con_n = TRANS ? d.m1 : d.n1;
    const int32_t* out_idx = idx + (TRANS ? d.cols_off : d.rows_off);
    const int32_t* con_idx = idx + (TRANS ? d.rows_off : d.cols_off);
    const float* P = pin + (TRANS ? d.y_off : d.z_off);
    float* O = pout + (TRANS ? d.z_off : d.y_off);
    const int t = threadIdx.x;
    const int orow = t >> 2, cc0 = (t & 3) * 8;
    float acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = 0.f;
    for (int k0 = 0; k0 < con_n; k0 += 32) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            int id = t + 128 * e;
            int o, c;
            if (TRANS) { o = id & 31; c = id >> 5; } else { o = id >> 5; c = id & 31; }
            int go = it.o0 + o, gc = k0 + c;
            float v = 0.f;
            if (go < out_n && gc < con_n)
                v = TRANS ? entry(g, con_idx[gc], out_idx[go]) : entry(g, out_idx[go], con_idx[gc]);
            As[o][c] = v;
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            int id = t + 128 * e;
            int kk = id & 31, col = id >> 5;
            int gk = k0 + kk, gcol = it.c0 + col;
            float v = 0.f;
            if (gk < con_n && gcol < d.ell) {
                if (RANDOM) {
                    // continuous uniform(-1, 1): a +-1 sketch of a few columns is
                    // singular with non-negligible probability and loses directions
                    uint64_t h = splitmix64(d.seed ^ ((uint64_t)gk * 0x9E3779B97F4A7C15ull) ^ ((uint64_t)gcol << 40));
                    v = ((float)(h >> 40) + 0.5f) * (2.0f / 16777216.0f) - 1.0f;
                } else {
                    v = P[(int64_t)gcol * con_n + gk];
                }
            }
            Ps[kk][col] = v;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            float a = As[orow][kk];
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] = fmaf(a, Ps[kk][cc0 + j], acc[j]);
        }
        __syncthreads();
    }
    int go = it.o0 + orow;
    if (go < out_n)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            int col = it.c0 + cc0 + j;
            if (col < d.ell) O[(int64_t)col * out_n + go] = acc[j];
        }
}

__device__ __forceinline__ float block_sum(float v, float* red) {
    // 256 threads
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    float s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.f;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[32] = s;
    __syncthreads();
    return red[32];
}

// Modified Gram-Schmidt with one re-orthogonalisation pass, one CTA (256
// threads) per probe panel (rows x ell, column-major).  Columns that lose
// all but 1e-6 of their norm are set to zero (rank deficiency).  WANT_R
// records R (ell x ell, column-major, upper triangle) so panel = Q R.
template <bool WANT_R>
__global__ void __launch_bounds__(256) k_orth(const ProbeDesc* __restrict__ pd, float* __restrict__ pan,
                                              float* __restrict__ small, int which /*0: y panel, 1: z panel*/) {
    __shared__ float red[33];
    const ProbeDesc d = pd[blockIdx.x];
    const int rows = which == 0 ? d.m1 : d.n1;
    float* Pm = pan + (which == 0 ? d.y_off : d.z_off);
    float* R = small + d.s_off;
    const int ell = d.ell;
    if (WANT_R)
        for (int i = threadIdx.x; i < ell * ell; i += blockDim.x) R[i] = 0.f;
    __syncthreads();
    for (int c = 0; c < ell; ++c) {
        float* yc = Pm + (int64_t)c * rows;
        float n0 = 0.f;
        for (int r = threadIdx.x; r < rows; r += blockDim.x) n0 += yc[r] * yc[r];
        n0 = block_sum(n0, red);
        for (int pass = 0; pass < 2; ++pass)
            for (int p = 0; p < c; ++p) {
                const float* qp = Pm + (int64_t)p * rows;
                float dd = 0.f;
                for (int r = threadIdx.x; r < rows; r += blockDim.x) dd += qp[r] * yc[r];
                dd = block_sum(dd, red);
                for (int r = threadIdx.x; r < rows; r += blockDim.x) yc[r] -= dd * qp[r];
                if (WANT_R && threadIdx.x == 0) R[(int64_t)c * ell + p] += dd;
                __syncthreads();
            }
        float nn = 0.f;
        for (int r = threadIdx.x; r < rows; r += blockDim.x) nn += yc[r] * yc[r];
        nn = block_sum(nn, red);
        float nrm = sqrtf(nn);
        bool keep = nrm > 1e-6f * sqrtf(n0) && nrm > 0.f;
        float inv = keep ? 1.f / nrm : 0.f;
        for (int r = threadIdx.x; r < rows; r += blockDim.x) yc[r] *= inv;
        if (WANT_R && threadIdx.x == 0) R[(int64_t)c * ell + c] = keep ? nrm : 0.f;
        __syncthreads();
    }
}

// One-sided Jacobi SVD of M = R^T (ell x ell) in shared memory, one CTA of
// 512 threads per probe, round-robin pair ordering, one warp per pair.  On
// exit small[s_off] holds M W (column-major; column norms = singular
// values), small[s_off + ell^2] holds W, small[s_off + 2 ell^2 ..] the
// column norms.
__global__ void __launch_bounds__(512) k_small_svd(const ProbeDesc* __restrict__ pd, float* __restrict__ small) {
    extern __shared__ float sm[];
    const ProbeDesc d = pd[blockIdx.x];
    const int ell = d.ell;
    const int L = ell + (ell & 1);  // padded to even
    float* M = sm;                  // L x L column-major
    float* W = sm + L * L;
    __shared__ int s_rot;
    __shared__ int s_perm[kMaxEll + 1];
    float* R = small + d.s_off;
    for (int i = threadIdx.x; i < L * L; i += blockDim.x) {
        int col = i / L, row = i % L;
        // M[row][col] = R[col][row]; R column-major: R[(row) * ell + col] is R[col][row]
        float v = 0.f;
        if (row < ell && col < ell) v = R[(int64_t)row * ell + col];
        M[i] = v;
        W[i] = (row == col) ? 1.f : 0.f;
    }
    for (int i = threadIdx.x; i < L; i += blockDim.x) s_perm[i] = i;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int sweep = 0; sweep < 30; ++sweep) {
        if (threadIdx.x == 0) s_rot = 0;
        __syncthreads();
        for (int round = 0; round < L - 1; ++round) {
            for (int k = warp; k < L / 2; k += nw) {
                int p = s_perm[k], q = s_perm[L - 1 - k];
                if (p > q) { int tt = p; p = q; q = tt; }
                float* mp = M + p * L;
                float* mq = M + q * L;
                float al = 0.f, be = 0.f, ga = 0.f;
                for (int r = lane; r < L; r += 32) {
                    float x = mp[r], y = mq[r];
                    al += x * x; be += y * y; ga += x * y;
                }
                for (int o = 16; o > 0; o >>= 1) {
                    al += __shfl_xor_sync(0xffffffffu, al, o);
                    be += __shfl_xor_sync(0xffffffffu, be, o);
                    ga += __shfl_xor_sync(0xffffffffu, ga, o);
                }
                if (fabsf(ga) > 1e-7f * sqrtf(al * be) && al > 0.f && be > 0.f) {
                    float zeta = (be - al) / (2.f * ga);
                    float tn = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
                    float cs = rsqrtf(1.f + tn * tn), sn = cs * tn;
                    float* wp = W + p * L;
                    float* wq = W + q * L;
                    for (int r = lane; r < L; r += 32) {
                        float x = mp[r], y = mq[r];
                        mp[r] = cs * x - sn * y;
                        mq[r] = sn * x + cs * y;
                        float u = wp[r], v = wq[r];
                        wp[r] = cs * u - sn * v;
                        wq[r] = sn * u + cs * v;
                    }
                    if (lane == 0) s_rot = 1;
                }
            }
            __syncthreads();
            // rotate the tournament: keep s_perm[0], shift the rest
            if (threadIdx.x == 0) {
                int last = s_perm[L - 1];
                for (int i = L - 1; i > 1; --i) s_perm[i] = s_perm[i - 1];
                s_perm[1] = last;
            }
            __syncthreads();
        }
        if (!s_rot) break;
        __syncthreads();
    }
    float* outM = small + d.s_off;
    float* outW = small + d.s_off + (int64_t)ell * ell;
    float* sig = small + d.s_off + 2 * (int64_t)ell * ell;
    for (int i = threadIdx.x; i < ell * ell; i += blockDim.x) {
        int col = i / ell, row = i % ell;
        outM[i] = M[col * L + row];
        outW[i] = W[col * L + row];
    }
    __syncthreads();
    for (int c = warp; c < ell; c += nw) {
        float s = 0.f;
        for (int r = lane; r < ell; r += 32) s += M[c * L + r] * M[c * L + r];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) sig[c] = sqrtf(s);
    }
}

// Factor formation for accepted ranks: U'(m1 x q) = Q (MW)[:, sel],
// V'(n1 x q) = Q_Z W[:, sel]; row-major outputs into the staging pool.
struct FactorDesc {
    int32_t probe, q;
    int64_t sel_off;   // q selected column indices
    int64_t u_off;     // staging offset of U' (then V' follows)
};

__global__ void k_form_factors(const ProbeDesc* __restrict__ pd, const FactorDesc* __restrict__ fd,
                               const int32_t* __restrict__ sel, const float* __restrict__ Y,
                               const float* __restrict__ Z, const float* __restrict__ small,
                               float* __restrict__ stage) {
    const FactorDesc f = fd[blockIdx.x];
    const ProbeDesc d = pd[f.probe];
    const int ell = d.ell;
    const float* MW = small + d.s_off;
    const float* Wm = small + d.s_off + (int64_t)ell * ell;
    int64_t tot = (int64_t)(d.m1 + d.n1) * f.q;
    for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
        int64_t r = e / f.q;
        int tcol = (int)(e - r * f.q);
        int col = sel[f.sel_off + tcol];
        float s = 0.f;
        if (r < d.m1) {
            const float* Q = Y + d.y_off;
            for (int c = 0; c < ell; ++c) s = fmaf(Q[(int64_t)c * d.m1 + r], MW[(int64_t)col * ell + c], s);
        } else {
            int64_t rr = r - d.m1;
            const float* QZ = Z + d.z_off;
            for (int c = 0; c < ell; ++c) s = fmaf(QZ[(int64_t)c * d.n1 + rr], Wm[(int64_t)col * ell + c], s);
        }
        stage[f.u_off + e] = s;
    }
}

// ------------------------------------------------------------ FP64 truncation check
// For an accepted q-term factorisation U' V'^T of a block A (compacted rows
// and columns), the truncation criterion of Algorithm 3 is
// sigma_{q+1}(A) < tol sigma_1(A); by Eckart-Young sigma_{q+1}(A) is the
// spectral norm of A - A_q, so the check estimates ||A - U' V'^T||_2 and
// ||A||_2 by power iteration on E^T E and A^T A (E = A - U' V'^T) from one
// seeded start, with every product and sum in FP64 (entries as assembly
// evaluates them), and accepts iff the first <= tol x the second.  A
// failed check sends the block back to Algorithm 3's rank doubling.
constexpr int kVerifyIters = 8;
// Power iteration approaches both norms from below; the error's estimate
// must clear tol x ||A|| by this factor, which covers its shortfall.
constexpr double kVerifyMargin = 0.9;
// ranks a candidate may add, one at a time, after a failed check
constexpr int kVerifyRaise = 4;

struct VerDesc {
    int32_t probe, q;
    int64_t u_off;  // U' (m1 x q, row-major) in the staging buffer; V' (n1 x q) follows
    int64_t s_off;  // FP64 scratch: xE, xA (n1 each), yE, yA (m1 each), t (q)
    uint64_t seed;
};

struct VerItem {
    int32_t v, o0;  // candidate, first output row (32 per item)
};

__device__ __forceinline__ double block_sum_d(double v, double* red) {
    // 256 threads
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[32] = s;
    __syncthreads();
    return red[32];
}

// out[k] = sum_r Fm[r q + k] x[r], k < q (Fm row-major rows x q, FP32; FP64 sums)
__device__ void ver_tdot(const float* Fm, int rows, int q, const double* x, double* out, double* red) {
    for (int k = 0; k < q; ++k) {
        double a = 0.0;
        for (int r = threadIdx.x; r < rows; r += blockDim.x) a += (double)Fm[(int64_t)r * q + k] * x[r];
        a = block_sum_d(a, red);
        if (threadIdx.x == 0) out[k] = a;
    }
}

// Start: xE = xA = a seeded uniform(-1, 1) vector, normalised; t = V'^T xE.
__global__ void __launch_bounds__(256) k_ver_start(const ProbeDesc* __restrict__ pd, const VerDesc* __restrict__ vd,
                                                   const float* __restrict__ stage, double* __restrict__ sc) {
    __shared__ double red[33];
    const VerDesc v = vd[blockIdx.x];
    const ProbeDesc d = pd[v.probe];
    double* xE = sc + v.s_off;
    double* xA = xE + d.n1;
    double* t = xA + 2 * (int64_t)d.m1 + d.n1;
    double nn = 0.0;
    for (int j = threadIdx.x; j < d.n1; j += blockDim.x) {
        const uint64_t h = splitmix64(v.seed ^ ((uint64_t)j * 0x9E3779B97F4A7C15ull));
        const double r = ((double)(h >> 11) + 0.5) * (2.0 / 9007199254740992.0) - 1.0;
        xE[j] = r;
        nn += r * r;
    }
    nn = block_sum_d(nn, red);
    const double inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
    for (int j = threadIdx.x; j < d.n1; j += blockDim.x) {
        xE[j] *= inv;
        xA[j] = xE[j];
    }
    __syncthreads();
    ver_tdot(stage + v.u_off + (int64_t)d.m1 * v.q, d.n1, v.q, xE, t, red);
}

// TRANS = false: yE = A xE - U' t, yA = A xA; TRANS = true: xE = A^T yE - V' t,
// xA = A^T yA.  One CTA (128 threads) per 32 output rows; entries in tiles
// of 32 x 32, four partial sums per output.
template <bool TRANS>
__global__ void __launch_bounds__(128) k_ver_pass(Geo g, const ProbeDesc* __restrict__ pd,
                                                  const VerDesc* __restrict__ vd, const VerItem* __restrict__ items,
                                                  const int32_t* __restrict__ idx, const float* __restrict__ stage,
                                                  double* __restrict__ sc) {
    __shared__ float As[32][33];
    __shared__ double vs[2][32];
    __shared__ double red[4][2][32];
    const VerItem it = items[blockIdx.x];
    const VerDesc v = vd[it.v];
    const ProbeDesc d = pd[v.probe];
    const int out_n = TRANS ? d.n1 : d.m1;
    const int con_n = TRANS ? d.m1 : d.n1;
    const int32_t* out_idx = idx + (TRANS ? d.cols_off : d.rows_off);
    const int32_t* con_idx = idx + (TRANS ? d.rows_off : d.cols_off);
    double* xE = sc + v.s_off;
    double* xA = xE + d.n1;
    double* yE = xA + d.n1;
    double* yA = yE + d.m1;
    const double* tq = yA + d.m1;
    const double* inE = TRANS ? yE : xE;
    const double* inA = TRANS ? yA : xA;
    double* outE = TRANS ? xE : yE;
    double* outA = TRANS ? xA : yA;
    const float* Fc = stage + v.u_off + (TRANS ? (int64_t)d.m1 * v.q : 0);  // the correction's factor
    const int t = threadIdx.x, row = t & 31, part = t >> 5;
    double accE = 0.0, accA = 0.0;
    for (int k0 = 0; k0 < con_n; k0 += 32) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int id = t + 128 * e;
            int o, c;
            if (TRANS) { o = id & 31; c = id >> 5; } else { o = id >> 5; c = id & 31; }
            const int go = it.o0 + o, gc = k0 + c;
            float a = 0.f;
            if (go < out_n && gc < con_n)
                a = TRANS ? entry(g, con_idx[gc], out_idx[go]) : entry(g, out_idx[go], con_idx[gc]);
            As[o][c] = a;
        }
        if (t < 64) {
            const int gk = k0 + (t & 31);
            vs[t >> 5][t & 31] = gk < con_n ? (t < 32 ? inE : inA)[gk] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = part * 8; kk < part * 8 + 8; ++kk) {
            const double a = (double)As[row][kk];
            accE = fma(a, vs[0][kk], accE);
            accA = fma(a, vs[1][kk], accA);
        }
        __syncthreads();
    }
    red[part][0][row] = accE;
    red[part][1][row] = accA;
    __syncthreads();
    if (t < 32) {
        const int go = it.o0 + t;
        if (go < out_n) {
            double sE = red[0][0][t] + red[1][0][t] + red[2][0][t] + red[3][0][t];
            const double sA = red[0][1][t] + red[1][1][t] + red[2][1][t] + red[3][1][t];
            for (int k = 0; k < v.q; ++k) sE -= (double)Fc[(int64_t)go * v.q + k] * tq[k];
            outE[go] = sE;
            outA[go] = sA;
        }
    }
}

// t = U'^T yE
__global__ void __launch_bounds__(256) k_ver_ut(const ProbeDesc* __restrict__ pd, const VerDesc* __restrict__ vd,
                                                const float* __restrict__ stage, double* __restrict__ sc) {
    __shared__ double red[33];
    const VerDesc v = vd[blockIdx.x];
    const ProbeDesc d = pd[v.probe];
    double* yE = sc + v.s_off + 2 * (int64_t)d.n1;
    ver_tdot(stage + v.u_off, d.m1, v.q, yE, yE + 2 * (int64_t)d.m1, red);
}

// After a T pass xE = E^T E x, xA = A^T A x for the previous unit x: record
// their norms (estimates of sigma_max^2), normalise, and form t = V'^T xE.
__global__ void __launch_bounds__(256) k_ver_norm(const ProbeDesc* __restrict__ pd, const VerDesc* __restrict__ vd,
                                                  const float* __restrict__ stage, double* __restrict__ sc,
                                                  double* __restrict__ lam) {
    __shared__ double red[33];
    const VerDesc v = vd[blockIdx.x];
    const ProbeDesc d = pd[v.probe];
    double* xE = sc + v.s_off;
    double* xA = xE + d.n1;
    double* t = xA + 2 * (int64_t)d.m1 + d.n1;
    double nE = 0.0, nA = 0.0;
    for (int j = threadIdx.x; j < d.n1; j += blockDim.x) {
        nE += xE[j] * xE[j];
        nA += xA[j] * xA[j];
    }
    nE = sqrt(block_sum_d(nE, red));
    nA = sqrt(block_sum_d(nA, red));
    if (threadIdx.x == 0) {
        lam[2 * blockIdx.x] = nE;
        lam[2 * blockIdx.x + 1] = nA;
    }
    const double iE = nE > 0.0 ? 1.0 / nE : 0.0, iA = nA > 0.0 ? 1.0 / nA : 0.0;
    for (int j = threadIdx.x; j < d.n1; j += blockDim.x) {
        xE[j] *= iE;
        xA[j] *= iA;
    }
    __syncthreads();
    ver_tdot(stage + v.u_off + (int64_t)d.m1 * v.q, d.n1, v.q, xE, t, red);
}

// ------------------------------------------------------------ packing
struct PackDesc {
    int32_t kind, r0, m, c0, n;
    int64_t off_val, off_aux;
    int64_t stage_off;  // SVD: staging offset
    int32_t q, m1, n1;
    int64_t lists_off;  // SVD: rows/cols in the probe index list
};

// dense: one CTA per block.  The block's rows that fall in one row tile
// [rs, re) form a column-major slab at off_val + (rs - r0) * n, so the
// multiply reads it with one lane per row and coalesced loads: element
// (row, c) is at slab + c * (re - rs) + (row - rs).
__global__ void k_pack_dense(Geo g, const PackDesc* __restrict__ pk, const int32_t* __restrict__ tile_of_row,
                             const int32_t* __restrict__ tile_first, const int32_t* __restrict__ tile_count,
                             float* __restrict__ val) {
    const PackDesc d = pk[blockIdx.x];
    for (int64_t e = threadIdx.x; e < (int64_t)d.m * d.n; e += blockDim.x) {
        const int c = (int)(e / d.m), r = (int)(e - (int64_t)c * d.m);  // consecutive threads: consecutive rows
        const int row = d.r0 + r;
        const int t = tile_of_row[row];
        const int rs = max(d.r0, tile_first[t]), re = min(d.r0 + d.m, tile_first[t] + tile_count[t]);
        val[d.off_val + (int64_t)(rs - d.r0) * d.n + (int64_t)c * (re - rs) + (row - rs)] = entry(g, row, d.c0 + c);
    }
}

// CSR: one CTA per block: row counts, exclusive scan, then the entries.
__global__ void k_pack_csr(Geo g, const PackDesc* __restrict__ pk, float* __restrict__ val, int32_t* __restrict__ aux) {
    const PackDesc d = pk[blockIdx.x];
    int32_t* rowptr = aux + d.off_aux;
    int32_t* cols = aux + d.off_aux + d.m + 1;
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int64_t w0 = d.c0 >> 5, w1 = (int64_t)(d.c0 + d.n - 1) >> 5;
    // counts into rowptr[r+1]
    for (int r = warp; r < d.m; r += nw) {
        const uint32_t* row = g.bits + (int64_t)(d.r0 + r) * g.ldw;
        int cnt = 0;
        for (int64_t w = w0 + lane; w <= w1; w += 32) {
            uint32_t x = row[w];
            int lo = (int)(d.c0 > w * 32 ? (int64_t)d.c0 : w * 32) - (int)(w * 32);
            int hi = (int)((int64_t)(d.c0 + d.n) < w * 32 + 32 ? (int64_t)(d.c0 + d.n) : w * 32 + 32) - (int)(w * 32);
            uint32_t mask = (hi >= 32 ? 0xffffffffu : ((1u << hi) - 1u)) & ~((1u << lo) - 1u);
            cnt += __popc(x & mask);
        }
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        if (lane == 0) rowptr[r + 1] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        rowptr[0] = 0;
        for (int r = 0; r < d.m; ++r) rowptr[r + 1] += rowptr[r];
    }
    __syncthreads();
    for (int r = warp; r < d.m; r += nw) {
        const uint32_t* row = g.bits + (int64_t)(d.r0 + r) * g.ldw;
        int base = rowptr[r];
        for (int64_t wb = w0; wb <= w1; wb += 32) {
            int64_t w = wb + lane;
            uint32_t x = 0;
            if (w <= w1) {
                x = row[w];
                int lo = (int)(d.c0 > w * 32 ? (int64_t)d.c0 : w * 32) - (int)(w * 32);
                int hi = (int)((int64_t)(d.c0 + d.n) < w * 32 + 32 ? (int64_t)(d.c0 + d.n) : w * 32 + 32) - (int)(w * 32);
                uint32_t mask = (hi >= 32 ? 0xffffffffu : ((1u << hi) - 1u)) & ~((1u << lo) - 1u);
                x &= mask;
            }
            int c = __popc(x);
            int incl = c;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            int pos = base + incl - c;
            while (x) {
                int bpos = __ffs(x) - 1;
                x &= x - 1;
                int j = (int)(w * 32 + bpos);
                cols[pos] = j;
                val[d.off_val + pos] = entry(g, d.r0 + r, j);
                ++pos;
            }
            base += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

__global__ void k_pack_svd(const PackDesc* __restrict__ pk, const int32_t* __restrict__ lists,
                           const float* __restrict__ stage, float* __restrict__ val, int32_t* __restrict__ aux) {
    const PackDesc d = pk[blockIdx.x];
    int64_t nv = (int64_t)(d.m1 + d.n1) * d.q;
    for (int64_t e = threadIdx.x; e < nv; e += blockDim.x) val[d.off_val + e] = stage[d.stage_off + e];
    for (int e = threadIdx.x; e < d.m1 + d.n1; e += blockDim.x) aux[d.off_aux + e] = lists[d.lists_off + e];
}

__global__ void k_to_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

// FP8 E4M3 with one scale per block: scale = max|v| / 448.
__global__ void k_to_fp8(const HBlock* __restrict__ blocks, const float* __restrict__ x, __nv_fp8_e4m3* __restrict__ y,
                         float* __restrict__ scales) {
    __shared__ float red[33];
    const HBlock b = blocks[blockIdx.x];
    int64_t len = 0;
    if (b.kind == VF_BLK_DENSE) len = (int64_t)b.m * b.n;
    else if (b.kind == VF_BLK_CSR) len = b.m1;
    else if (b.kind == VF_BLK_SVD) len = (int64_t)(b.m1 + b.n1) * b.q;
    float mx = 0.f;
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) mx = fmaxf(mx, fabsf(x[b.off_val + i]));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
        red[32] = m > 0.f ? m / 448.f : 1.f;
        scales[blockIdx.x] = red[32];
    }
    __syncthreads();
    float inv = 1.f / red[32];
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) y[b.off_val + i] = __nv_fp8_e4m3(x[b.off_val + i] * inv);
}

// ============================================================ host DP
namespace {

// CSR bytes; blocks whose nonzeros overflow the int32 row pointers cannot be CSR
inline int64_t csr_bytes(int64_t m, int64_t nnz) {
    return nnz >= (int64_t(1) << 31) ? INT64_MAX / 4 : 8 * nnz + 4 * (m + 1);
}

struct Stats {
    int64_t nnz = 0;
    int32_t m1 = 0, n1 = 0;
};

struct DNode {
    int32_t I, J;
    int32_t kid_begin = 0, kid_end = 0;  // into kids
    int32_t height = 0;
    Stats st;
    int32_t kind = -1;
    int64_t bytes = 0;
    int32_t q = 0;
    // probe bookkeeping
    int64_t best_alt = 0;
    int64_t hier_bytes = 0;
    int32_t k = 0;           // current probe rank
    int32_t stage_slot = -1; // accepted factors in staging
    int64_t stage_off = -1;
    int64_t lists_off = -1;  // rows then cols in the persistent list pool
};

// a child reference: a DNode (>= 0) or an implicit leaf pair (-1 - pair index)
struct Kid {
    int64_t ref;
};

struct Builder {
    const vf_tree* t;
    const vf_assemble_opts* o;
    int64_t nleaves = 0;
    std::vector<int32_t> leaf_of_node_begin, leaf_of_node_end;  // leaf range per node
    std::vector<int32_t> leaf_first, leaf_count;
    std::vector<unsigned long long> rowmask, colmask;
    std::vector<int32_t> pnnz;
    std::vector<DNode> nodes;
    std::vector<Kid> kids;
    std::vector<int32_t> top;  // top-level DNode ids or leaf pair refs
    std::vector<Kid> top_refs;

    int64_t pair_index(int32_t a, int32_t b) const { return (int64_t)a * nleaves + b; }

    Stats rect_stats(int32_t I, int32_t J) const {
        Stats s;
        int32_t a0 = leaf_of_node_begin[I], a1 = leaf_of_node_end[I];
        int32_t b0 = leaf_of_node_begin[J], b1 = leaf_of_node_end[J];
        std::vector<unsigned long long> cm(b1 - b0, 0ull);
        for (int32_t a = a0; a < a1; ++a) {
            unsigned long long rm = 0;
            for (int32_t b = b0; b < b1; ++b) {
                int64_t p = pair_index(a, b);
                s.nnz += pnnz[p];
                rm |= rowmask[p];
                cm[b - b0] |= colmask[p];
            }
            s.m1 += __builtin_popcountll(rm);
        }
        for (auto x : cm) s.n1 += __builtin_popcountll(x);
        return s;
    }

    // tree positions of the nonzero rows and columns of block (I, J)
    void nz_lists(int32_t I, int32_t J, std::vector<int32_t>& rows, std::vector<int32_t>& cols) const {
        int32_t a0 = leaf_of_node_begin[I], a1 = leaf_of_node_end[I];
        int32_t b0 = leaf_of_node_begin[J], b1 = leaf_of_node_end[J];
        std::vector<unsigned long long> cm(b1 - b0, 0ull);
        for (int32_t a = a0; a < a1; ++a) {
            unsigned long long rm = 0;
            for (int32_t b = b0; b < b1; ++b) {
                int64_t p = pair_index(a, b);
                rm |= rowmask[p];
                cm[b - b0] |= colmask[p];
            }
            for (int r = 0; r < 64; ++r)
                if ((rm >> r) & 1ull) rows.push_back(leaf_first[a] + r);
        }
        for (int32_t b = b0; b < b1; ++b)
            for (int c = 0; c < 64; ++c)
                if ((cm[b - b0] >> c) & 1ull) cols.push_back(leaf_first[b] + c);
    }

    bool is_leaf_block(int32_t I, int32_t J) const {
        return (t->is_leaf(I) && t->is_leaf(J)) ||
               (int64_t)t->count[I] * t->count[J] < o->leaf_threshold;
    }

    // returns a Kid for the block (I, J), creating DNodes recursively
    Kid make(int32_t I, int32_t J) {
        if (t->is_leaf(I) && t->is_leaf(J)) {
            int32_t a = leaf_of_node_begin[I], b = leaf_of_node_begin[J];
            return Kid{-1 - pair_index(a, b)};
        }
        int32_t id = (int32_t)nodes.size();
        nodes.push_back(DNode{});
        nodes[id].I = I;
        nodes[id].J = J;
        if (is_leaf_block(I, J)) {
            nodes[id].height = 0;
            return Kid{id};
        }
        std::vector<int32_t> ki = t->is_leaf(I) ? std::vector<int32_t>{I} : t->kids[I];
        std::vector<int32_t> kj = t->is_leaf(J) ? std::vector<int32_t>{J} : t->kids[J];
        std::vector<Kid> mine;
        for (int32_t a : ki)
            for (int32_t b : kj) mine.push_back(make(a, b));
        int32_t h = 0;
        for (auto& k : mine) h = std::max(h, k.ref >= 0 ? nodes[k.ref].height + 1 : 1);
        nodes[id].kid_begin = (int32_t)kids.size();
        kids.insert(kids.end(), mine.begin(), mine.end());
        nodes[id].kid_end = (int32_t)kids.size();
        nodes[id].height = h;
        return Kid{id};
    }

    int32_t kid_kind(const Kid& k) const {
        if (k.ref >= 0) return nodes[k.ref].kind;
        int64_t p = -1 - k.ref;
        return leaf_pair_choice(p).first;
    }
    int64_t kid_bytes(const Kid& k) const {
        if (k.ref >= 0) return nodes[k.ref].bytes;
        return leaf_pair_choice(-1 - k.ref).second;
    }
    std::pair<int32_t, int64_t> leaf_pair_choice(int64_t p) const {
        int64_t a = p / nleaves, b = p - a * nleaves;
        return leaf_choice(leaf_count[a], leaf_count[b], pnnz[p]);
    }
    static std::pair<int32_t, int64_t> leaf_choice(int64_t m, int64_t n, int64_t nnz) {
        if (nnz == 0) return {VF_BLK_ZERO, 0};
        int64_t bd = 4 * m * n, bc = csr_bytes(m, nnz);
        return bd <= bc ? std::make_pair((int32_t)VF_BLK_DENSE, bd) : std::make_pair((int32_t)VF_BLK_CSR, bc);
    }
};

int32_t ell_for(int32_t k, int32_t m1, int32_t n1) {
    int32_t over = std::min(32, k / 2 + 8);
    int32_t ell = std::min(k + over, kMaxEll);
    return std::min(ell, std::min(m1, n1));
}

int64_t svd_bytes(int64_t q, int64_t m1, int64_t n1) { return 4 * q * (m1 + n1) + 4 * (m1 + n1); }

}  // namespace

// Runs the probe pipeline for a batch; returns sigma (sorted desc) per probe
// and keeps the panels for factor formation.
struct ProbeBatch {
    std::vector<ProbeDesc> pd;
    std::vector<int32_t> lists;  // rows then cols per probe
    dbuf<ProbeDesc> d_pd;
    dbuf<int32_t> d_lists;
    dbuf<float> Y, Z, small;
    int64_t ny = 0, nz = 0, ns = 0;
};

static vf_status build_panel_items(const std::vector<ProbeDesc>& pd, bool trans, std::vector<PanelItem>& items) {
    items.clear();
    for (size_t p = 0; p < pd.size(); ++p) {
        int out_n = trans ? pd[p].n1 : pd[p].m1;
        for (int o = 0; o < out_n; o += 32)
            for (int c = 0; c < pd[p].ell; c += 32) items.push_back(PanelItem{(int32_t)p, o, c, 0});
    }
    return VF_OK;
}

static vf_status run_probes(const Geo& g, ProbeBatch& B, int power_iters, cudaStream_t st) {
    const size_t np = B.pd.size();
    if (np == 0) return VF_OK;
    VF_TRY(B.d_pd.upload(B.pd));
    VF_TRY(B.d_lists.upload(B.lists));
    VF_TRY(B.Y.alloc(std::max<int64_t>(B.ny, 1)));
    VF_TRY(B.Z.alloc(std::max<int64_t>(B.nz, 1)));
    VF_TRY(B.small.alloc(std::max<int64_t>(B.ns, 1)));
    std::vector<PanelItem> it_a, it_t;
    build_panel_items(B.pd, false, it_a);
    build_panel_items(B.pd, true, it_t);
    dbuf<PanelItem> d_ia, d_it;
    VF_TRY(d_ia.upload(it_a));
    VF_TRY(d_it.upload(it_t));
    const unsigned na = (unsigned)it_a.size(), nt = (unsigned)it_t.size();
    // Y = A Omega
    k_apanel<false, true><<<na, 128, 0, st>>>(g, B.d_pd.p, d_ia.p, B.d_lists.p, B.Z.p, B.Y.p);
    VF_TRY_CUDA(cudaGetLastError());
    k_orth<false><<<(unsigned)np, 256, 0, st>>>(B.d_pd.p, B.Y.p, B.small.p, 0);
    for (int it = 0; it < power_iters; ++it) {
        k_apanel<true, false><<<nt, 128, 0, st>>>(g, B.d_pd.p, d_it.p, B.d_lists.p, B.Y.p, B.Z.p);
        k_orth<false><<<(unsigned)np, 256, 0, st>>>(B.d_pd.p, B.Z.p, B.small.p, 1);
        k_apanel<false, false><<<na, 128, 0, st>>>(g, B.d_pd.p, d_ia.p, B.d_lists.p, B.Z.p, B.Y.p);
        k_orth<false><<<(unsigned)np, 256, 0, st>>>(B.d_pd.p, B.Y.p, B.small.p, 0);
    }
    k_apanel<true, false><<<nt, 128, 0, st>>>(g, B.d_pd.p, d_it.p, B.d_lists.p, B.Y.p, B.Z.p);
    k_orth<true><<<(unsigned)np, 256, 0, st>>>(B.d_pd.p, B.Z.p, B.small.p, 1);
    int maxell = 0;
    for (auto& p : B.pd) maxell = std::max(maxell, p.ell);
    int L = maxell + (maxell & 1);
    size_t smem = 2 * (size_t)L * L * sizeof(float);
    VF_TRY_CUDA(cudaFuncSetAttribute(k_small_svd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_small_svd<<<(unsigned)np, 512, smem, st>>>(B.d_pd.p, B.small.p);
    VF_TRY_CUDA(cudaGetLastError());
    return VF_OK;
}

// The FP64 truncation check of the factorisations fds (formed into stage)
// of batch B: ok[f] = 1 iff ||A - U' V'^T||_2 <= tol ||A||_2 (estimates);
// est[2 f], est[2 f + 1] = the two norms.
static vf_status verify_factors(const Geo& g, const ProbeBatch& B, const std::vector<FactorDesc>& fds,
                                const float* stage, double tol, uint64_t seed, std::vector<uint8_t>& ok,
                                std::vector<double>& est, cudaStream_t st) {
    const size_t nv = fds.size();
    ok.assign(nv, 1);
    est.assign(2 * nv, 0.0);
    if (nv == 0) return VF_OK;
    std::vector<VerDesc> vd(nv);
    std::vector<VerItem> itn, itt;
    int64_t ns = 0;
    for (size_t f = 0; f < nv; ++f) {
        const ProbeDesc& p = B.pd[fds[f].probe];
        vd[f] = VerDesc{fds[f].probe, fds[f].q, fds[f].u_off, ns, splitmix64(seed ^ (0xC0FFEEull + f))};
        ns += 2 * (int64_t)(p.m1 + p.n1) + fds[f].q;
        for (int32_t o = 0; o < p.m1; o += 32) itn.push_back(VerItem{(int32_t)f, o});
        for (int32_t o = 0; o < p.n1; o += 32) itt.push_back(VerItem{(int32_t)f, o});
    }
    dbuf<VerDesc> dvd;
    dbuf<VerItem> din, dit;
    dbuf<double> sc, lam;
    VF_TRY(dvd.upload(vd));
    VF_TRY(din.upload(itn));
    VF_TRY(dit.upload(itt));
    VF_TRY(sc.alloc(std::max<int64_t>(ns, 1)));
    VF_TRY(lam.alloc(2 * (int64_t)nv));
    k_ver_start<<<(unsigned)nv, 256, 0, st>>>(B.d_pd.p, dvd.p, stage, sc.p);
    VF_CHECK(!itn.empty() && !itt.empty(), VF_E_INVAL, "truncation check: empty candidate");
    for (int it = 0; it < kVerifyIters; ++it) {
        k_ver_pass<false><<<(unsigned)itn.size(), 128, 0, st>>>(g, B.d_pd.p, dvd.p, din.p, B.d_lists.p, stage, sc.p);
        k_ver_ut<<<(unsigned)nv, 256, 0, st>>>(B.d_pd.p, dvd.p, stage, sc.p);
        k_ver_pass<true><<<(unsigned)itt.size(), 128, 0, st>>>(g, B.d_pd.p, dvd.p, dit.p, B.d_lists.p, stage, sc.p);
        k_ver_norm<<<(unsigned)nv, 256, 0, st>>>(B.d_pd.p, dvd.p, stage, sc.p, lam.p);
    }
    VF_TRY_CUDA(cudaGetLastError());
    VF_TRY_CUDA(cudaMemcpyAsync(est.data(), lam.p, 2 * nv * sizeof(double), cudaMemcpyDeviceToHost, st));
    VF_TRY_CUDA(cudaStreamSynchronize(st));
    for (size_t f = 0; f < nv; ++f) {
        est[2 * f] = std::sqrt(est[2 * f]);  // sigma_max(E), sigma_max(A)
        est[2 * f + 1] = std::sqrt(est[2 * f + 1]);
        ok[f] = est[2 * f] <= kVerifyMargin * tol * est[2 * f + 1] ? 1 : 0;
    }
    return VF_OK;
}

}  // namespace vf

using namespace vf;


extern "C" vf_status vf_assemble(const vf_mesh* m, const vf_tree* t, const vf_assemble_opts* opts_in, vf_hmat** out,
                                 vf_assemble_stats* stats_out) {
    clear_error();
    VF_CHECK(m && t && out, VF_E_INVAL, "vf_assemble: null argument");
    VF_CHECK(t->nf == m->nf, VF_E_INVAL, "vf_assemble: tree and mesh sizes differ");
    *out = nullptr;
    vf_assemble_opts o{};
    o.tol = 1e-3;
    o.leaf_threshold = 4096;
    o.k0 = 8;
    o.k_max = 128;
    o.power_iters = 2;
    o.verify = 1;
    o.precisions = (1u << VF_PREC_FP32) | (1u << VF_PREC_BF16);
    o.seed = 12345;
    o.storage = 0;
    if (opts_in) {
        o = *opts_in;
        if (o.leaf_threshold <= 0) o.leaf_threshold = 4096;
        if (o.k0 <= 0) o.k0 = 8;
        if (o.k_max <= 0) o.k_max = 128;
        if (o.power_iters < 0) o.power_iters = 2;
    }
    VF_CHECK(o.tol > 0 && o.tol < 1, VF_E_INVAL, "vf_assemble: tol must be in (0, 1)");
    VF_CHECK(o.k_max <= 128, VF_E_INVAL, "vf_assemble: k_max above 128 is not supported");
    VF_CHECK(o.storage >= 0 && o.storage <= 2, VF_E_INVAL, "vf_assemble: storage must be 0, 1 or 2");
    const int64_t n = m->nf;
    for (size_t k = 0; k < t->first.size(); ++k)
        VF_CHECK(!t->is_leaf((int)k) || t->count[k] <= 64, VF_E_INVAL,
                 "vf_assemble: tree leaf %zu holds %d facets (> 64); lower leaf_size or raise max_depth", k,
                 t->count[k]);
    device_guard dg(m->device);
    cudaStream_t st = 0;
    double t0 = now_seconds();
    vf_assemble_stats S{};

    auto H = std::make_unique<vf_hmat>();
    H->device = m->device;
    H->nf = n;
    H->tol = o.tol;
    H->tree_kind = t->kind;
    H->h_perm = t->perm;
    VF_TRY(H->perm.upload(t->perm));
    {
        std::vector<int32_t> ip(n);
        for (int64_t k = 0; k < n; ++k) ip[t->perm[k]] = (int32_t)k;
        VF_TRY(H->iperm.upload(ip));
    }
    // ---------------- tree-order geometry and visibility bits
    dbuf<float4> xa, nv;
    VF_TRY(xa.alloc(n));
    VF_TRY(nv.alloc(n));
    k_tree_geom<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(H->perm.p, m->c3.p, m->area.p, m->nrm.p, n, xa.p, nv.p);
    const int64_t ldw = ceil_div(n, 32);
    dbuf<uint32_t> bits;
    VF_TRY(bits.alloc(n * ldw));
    VF_TRY(visibility_bits(m, H->perm.p, n, bits.p, ldw, st));
    VF_TRY_CUDA(cudaStreamSynchronize(st));
    double t1 = now_seconds();
    S.t_visibility = t1 - t0;
    Geo g{xa.p, nv.p, bits.p, ldw, (float)(m->unit / 3.0)};

    // ---------------- leaves and leaf-pair statistics
    Builder Bd;
    Bd.t = t;
    Bd.o = &o;
    const int32_t nnodes = (int32_t)t->first.size();
    Bd.leaf_of_node_begin.assign(nnodes, 0);
    Bd.leaf_of_node_end.assign(nnodes, 0);
    {
        // leaves in preorder = tree-position order; a node's leaves are contiguous
        std::vector<int32_t> leaf_index(nnodes, -1);
        for (int32_t k = 0; k < nnodes; ++k)
            if (t->is_leaf(k)) {
                leaf_index[k] = (int32_t)Bd.leaf_first.size();
                Bd.leaf_first.push_back(t->first[k]);
                Bd.leaf_count.push_back(t->count[k]);
            }
        // postorder accumulation of leaf ranges (preorder ids: children > parent)
        for (int32_t k = nnodes - 1; k >= 0; --k) {
            if (t->is_leaf(k)) {
                Bd.leaf_of_node_begin[k] = leaf_index[k];
                Bd.leaf_of_node_end[k] = leaf_index[k] + 1;
            } else {
                Bd.leaf_of_node_begin[k] = Bd.leaf_of_node_begin[t->kids[k].front()];
                Bd.leaf_of_node_end[k] = Bd.leaf_of_node_end[t->kids[k].back()];
            }
        }
    }
    Bd.nleaves = (int64_t)Bd.leaf_first.size();
    const int64_t npairs = Bd.nleaves * Bd.nleaves;
    {
        dbuf<int32_t> dlf, dlc;
        VF_TRY(dlf.upload(Bd.leaf_first));
        VF_TRY(dlc.upload(Bd.leaf_count));
        Bd.rowmask.resize(npairs);
        Bd.colmask.resize(npairs);
        Bd.pnnz.resize(npairs);
        const int64_t chunk = 1 << 24;
        dbuf<unsigned long long> drm, dcm;
        dbuf<int32_t> dnz;
        VF_TRY(drm.alloc(std::min(chunk, npairs)));
        VF_TRY(dcm.alloc(std::min(chunk, npairs)));
        VF_TRY(dnz.alloc(std::min(chunk, npairs)));
        for (int64_t p0 = 0; p0 < npairs; p0 += chunk) {
            int64_t np = std::min(chunk, npairs - p0);
            k_leaf_pair_stats<<<(unsigned)ceil_div(np * 32, 256), 256, 0, st>>>(
                bits.p, ldw, dlf.p, dlc.p, Bd.nleaves, p0, np, drm.p, dcm.p, dnz.p);
            VF_TRY_CUDA(cudaGetLastError());
            VF_TRY_CUDA(cudaMemcpy(Bd.rowmask.data() + p0, drm.p, np * 8, cudaMemcpyDeviceToHost));
            VF_TRY_CUDA(cudaMemcpy(Bd.colmask.data() + p0, dcm.p, np * 8, cudaMemcpyDeviceToHost));
            VF_TRY_CUDA(cudaMemcpy(Bd.pnnz.data() + p0, dnz.p, np * 4, cudaMemcpyDeviceToHost));
        }
    }
    for (int64_t p = 0; p < npairs; ++p) S.nnz_visible += Bd.pnnz[p];

    std::vector<HBlock>& HB = H->h_blocks;
    std::vector<int32_t> hb_node;  // DNode id of each stored block (-1 for a leaf pair)
    std::vector<DNode>& N = Bd.nodes;
    std::vector<int32_t> lists_pool;                       // rows/cols of SVD candidates
    std::vector<std::unique_ptr<dbuf<float>>> stage_bufs;  // their factors
    struct StageRef { int32_t buf; int64_t off; };
    std::vector<StageRef> stage_ref;
    double t2 = now_seconds(), t3 = t2;
    if (o.storage != 0) {
        // the uncompressed F (dense) or Algorithm 1's CSR, one block per leaf pair
        for (int64_t a = 0; a < Bd.nleaves; ++a)
            for (int64_t bb = 0; bb < Bd.nleaves; ++bb) {
                int64_t p = Bd.pair_index((int32_t)a, (int32_t)bb);
                int32_t kind = o.storage == 1 ? VF_BLK_DENSE : VF_BLK_CSR;
                if (kind == VF_BLK_CSR && Bd.pnnz[p] == 0) { S.nblocks[VF_BLK_ZERO]++; continue; }
                HBlock blk{};
                blk.kind = kind;
                blk.I = blk.J = -1;
                blk.r0 = Bd.leaf_first[a];
                blk.m = Bd.leaf_count[a];
                blk.c0 = Bd.leaf_first[bb];
                blk.n = Bd.leaf_count[bb];
                blk.m1 = Bd.pnnz[p];
                S.nblocks[kind]++;
                HB.push_back(blk);
                hb_node.push_back(-1);
            }
        t3 = now_seconds();
        S.t_stats = t3 - t1;
    } else {
        // ---------------- block tree
        if (t->is_leaf(0)) {
            Bd.top_refs.push_back(Bd.make(0, 0));
        } else {
            for (int32_t a : t->kids[0])
                for (int32_t b : t->kids[0]) Bd.top_refs.push_back(Bd.make(a, b));
        }
        int32_t maxh = 0;
        for (auto& d : N) {
            d.st = Bd.rect_stats(d.I, d.J);
            maxh = std::max(maxh, d.height);
        }
        // per tree node: mean centroid, bounding-box diagonal and mean unit
        // normal (the predictor's features; FP64 from the snapped geometry)
        std::vector<double> ncen(3 * (size_t)nnodes, 0.0), ndiam(nnodes, 0.0), nnrm(3 * (size_t)nnodes, 0.0);
        {
            std::vector<double> hn;
            VF_TRY(m->nrm.download(hn));
            const double s = m->unit / 3.0;
            for (int32_t k = 0; k < nnodes; ++k) {
                double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
                for (int32_t pos = t->first[k]; pos < t->first[k] + t->count[k]; ++pos) {
                    const int32_t f = t->perm[pos];
                    for (int a = 0; a < 3; ++a) {
                        const double x = s * m->h_c3[3 * (size_t)f + a];
                        ncen[3 * (size_t)k + a] += x;
                        lo[a] = std::min(lo[a], x);
                        hi[a] = std::max(hi[a], x);
                        nnrm[3 * (size_t)k + a] += hn[3 * (size_t)f + a];
                    }
                }
                const double c = (double)std::max(t->count[k], 1);
                double d2 = 0;
                for (int a = 0; a < 3; ++a) {
                    ncen[3 * (size_t)k + a] /= c;
                    nnrm[3 * (size_t)k + a] /= c;
                    d2 += (hi[a] - lo[a]) * (hi[a] - lo[a]);
                }
                ndiam[k] = std::sqrt(d2);
            }
        }
        auto features = [&](const DNode& d, float* f) {
            const double mm = t->count[d.I], nn = t->count[d.J];
            const double* ci = &ncen[3 * (size_t)d.I];
            const double* cj = &ncen[3 * (size_t)d.J];
            const double* ni = &nnrm[3 * (size_t)d.I];
            const double* nj = &nnrm[3 * (size_t)d.J];
            const double dist = std::sqrt((ci[0] - cj[0]) * (ci[0] - cj[0]) + (ci[1] - cj[1]) * (ci[1] - cj[1]) +
                                          (ci[2] - cj[2]) * (ci[2] - cj[2]));
            f[0] = (float)std::log2(mm);
            f[1] = (float)std::log2(nn);
            f[2] = (float)(d.st.m1 / mm);
            f[3] = (float)(d.st.n1 / nn);
            f[4] = (float)((double)d.st.nnz / (mm * nn));
            f[5] = (float)(dist / std::max(ndiam[d.I] + ndiam[d.J], 1e-300));
            f[6] = (float)(ni[0] * nj[0] + ni[1] * nj[1] + ni[2] * nj[2]);
            f[7] = (float)std::sqrt(ni[0] * ni[0] + ni[1] * ni[1] + ni[2] * ni[2]);
            f[8] = (float)std::sqrt(nj[0] * nj[0] + nj[1] * nj[1] + nj[2] * nj[2]);
            f[9] = (float)d.height;
        };
        t2 = now_seconds();
        S.t_stats = t2 - t1;

        // ---------------- DP bottom-up by height
        stage_ref.assign(N.size(), StageRef{-1, -1});
        std::vector<int32_t> log_ids;  // probed candidates, in order (the probe log)

        for (int32_t h = 0; h <= maxh; ++h) {
            std::vector<int32_t> level;
            for (int32_t id = 0; id < (int32_t)N.size(); ++id)
                if (N[id].height == h) level.push_back(id);
            // alternatives
            std::vector<int32_t> pending;
            for (int32_t id : level) {
                DNode& d = N[id];
                int64_t mm = t->count[d.I], nn = t->count[d.J];
                if (h == 0) {
                    auto c = Builder::leaf_choice(mm, nn, d.st.nnz);
                    d.kind = c.first;
                    d.bytes = c.second;
                    continue;
                }
                if (d.st.nnz == 0) {
                    d.kind = VF_BLK_ZERO;
                    d.bytes = 0;
                    continue;
                }
                int64_t hb = 0;
                for (int32_t k = d.kid_begin; k < d.kid_end; ++k) hb += Bd.kid_bytes(Bd.kids[k]);
                d.hier_bytes = hb;
                int64_t bd = 4 * mm * nn, bc = csr_bytes(mm, d.st.nnz);
                d.best_alt = std::min(std::min(bd, bc), hb);
                // the SVD can only win if some q >= 1 has svd_bytes(q) < best_alt
                if (svd_bytes(1, d.st.m1, d.st.n1) < d.best_alt) {
                    d.k = std::min(o.k0, o.k_max);
                    pending.push_back(id);
                } else {
                    S.probes_skipped++;
                }
            }
            // the candidates' features; the predictor (if any) picks each
            // first probe rank or skips the probe
            const size_t log0 = log_ids.size();
            std::vector<int32_t> audit, skipped;
            std::vector<float> skipped_feat;
            {
                std::vector<float> fl(pending.size() * VF_PRED_NFEAT);
                for (size_t i = 0; i < pending.size(); ++i) features(N[pending[i]], &fl[i * VF_PRED_NFEAT]);
                std::vector<int32_t> keep;
                if (o.predictor && !pending.empty()) {
                    std::vector<int32_t> cls;
                    std::vector<float> prob;
                    VF_TRY(predictor_classify(o.predictor, fl, (int64_t)pending.size(), cls, prob));
                    std::vector<float> fk;
                    int64_t nskip = 0;
                    for (size_t i = 0; i < pending.size(); ++i) {
                        DNode& d = N[pending[i]];
                        if (cls[i] == VF_PRED_NCLASS - 1 && prob[i * VF_PRED_NCLASS + cls[i]] >= 0.9f) {
                            // every kAuditEvery-th predicted skip is probed anyway (an audit)
                            if (nskip++ % kAuditEvery == 0) {
                                audit.push_back(pending[i]);
                            } else {
                                S.probes_predicted_skip++;
                                skipped.push_back(pending[i]);
                                skipped_feat.insert(skipped_feat.end(), fl.begin() + i * VF_PRED_NFEAT,
                                                    fl.begin() + (i + 1) * VF_PRED_NFEAT);
                                continue;
                            }
                        }
                        if (cls[i] < VF_PRED_NCLASS - 1) d.k = std::min(std::max(o.k0, 8 << cls[i]), o.k_max);
                        keep.push_back(pending[i]);
                        fk.insert(fk.end(), fl.begin() + i * VF_PRED_NFEAT, fl.begin() + (i + 1) * VF_PRED_NFEAT);
                    }
                    pending.swap(keep);
                    fl.swap(fk);
                }
                log_ids.insert(log_ids.end(), pending.begin(), pending.end());
                H->h_probe_feat.insert(H->h_probe_feat.end(), fl.begin(), fl.end());
            }
            // probe rounds (k doubling, Algorithm 3)
            auto probe_rounds = [&](std::vector<int32_t>& pending) -> vf_status {
            while (!pending.empty()) {
                ProbeBatch B;
                std::vector<int32_t> who;
                for (int32_t id : pending) {
                    DNode& d = N[id];
                    ProbeDesc p{};
                    p.m1 = d.st.m1;
                    p.n1 = d.st.n1;
                    p.ell = ell_for(d.k, p.m1, p.n1);
                    p.rows_off = (int64_t)B.lists.size();
                    std::vector<int32_t> rows, cols;
                    Bd.nz_lists(d.I, d.J, rows, cols);
                    B.lists.insert(B.lists.end(), rows.begin(), rows.end());
                    p.cols_off = (int64_t)B.lists.size();
                    B.lists.insert(B.lists.end(), cols.begin(), cols.end());
                    p.y_off = B.ny;
                    B.ny += (int64_t)p.m1 * p.ell;
                    p.z_off = B.nz;
                    B.nz += (int64_t)p.n1 * p.ell;
                    p.s_off = B.ns;
                    B.ns += 2 * (int64_t)p.ell * p.ell + p.ell;
                    p.seed = splitmix64(o.seed ^ ((uint64_t)id << 20) ^ (uint64_t)d.k);
                    B.pd.push_back(p);
                    who.push_back(id);
                }
                VF_TRY(run_probes(g, B, o.power_iters, st));
                std::vector<float> hsmall(B.ns);
                VF_TRY_CUDA(cudaMemcpy(hsmall.data(), B.small.p, B.ns * 4, cudaMemcpyDeviceToHost));
                S.probes += (int64_t)who.size();
                std::vector<int32_t> next;
                std::vector<FactorDesc> fds;
                std::vector<int32_t> sel;
                std::vector<int32_t> fd_owner;
                std::vector<std::vector<int32_t>> orders(who.size());  // per probe: columns by singular value
                int64_t fstage = 0;
                for (size_t pi = 0; pi < who.size(); ++pi) {
                    DNode& d = N[who[pi]];
                    const ProbeDesc& p = B.pd[pi];
                    const float* sig = hsmall.data() + p.s_off + 2 * (int64_t)p.ell * p.ell;
                    std::vector<int32_t>& order = orders[pi];
                    order.resize(p.ell);
                    std::iota(order.begin(), order.end(), 0);
                    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sig[a] > sig[b]; });
                    float s1 = sig[order[0]];
                    bool full = p.ell == std::min(p.m1, p.n1);
                    int32_t trust = full ? p.ell : std::min(d.k, p.ell);
                    int32_t q = -1;
                    if (s1 > 0.f)
                        for (int32_t qq = 1; qq <= trust; ++qq) {
                            float nxt = qq < p.ell ? sig[order[qq]] : 0.f;
                            if (qq == trust && !full) break;  // sigma_{q+1} not trusted
                            if (nxt < (float)o.tol * s1) { q = qq; break; }
                        }
                    if (q < 0) {
                        int32_t k2 = 2 * d.k;
                        if (!full && k2 <= o.k_max && svd_bytes(d.k, d.st.m1, d.st.n1) < d.best_alt) {
                            d.k = k2;
                            next.push_back(who[pi]);
                        } else {
                            S.probes_failed++;
                        }
                        continue;
                    }
                    if (q > o.k_max || svd_bytes(q, d.st.m1, d.st.n1) >= d.best_alt) {
                        S.probes_failed += q > o.k_max ? 1 : 0;
                        continue;  // the SVD cannot win
                    }
                    d.q = q;
                    FactorDesc f{};
                    f.probe = (int32_t)pi;
                    f.q = q;
                    f.sel_off = (int64_t)sel.size();
                    for (int32_t k = 0; k < q; ++k) sel.push_back(order[k]);
                    f.u_off = fstage;
                    fstage += (int64_t)(p.m1 + p.n1) * q;
                    fds.push_back(f);
                    fd_owner.push_back(who[pi]);
                }
                // Form the accepted factorisations and check them.  A check can
                // fail when sigma_{q+1} sits just below tol sigma_1: the
                // randomized factors carry a little more than the optimal
                // truncation error.  Such a candidate retries with one more
                // rank from the same probe (up to kVerifyRaise times, while
                // the SVD still wins on bytes) before it goes back to the rank
                // doubling.
                for (int attempt = 0; !fds.empty(); ++attempt) {
                    auto buf = std::make_unique<dbuf<float>>();
                    VF_TRY(buf->alloc(fstage));
                    dbuf<FactorDesc> dfd;
                    dbuf<int32_t> dsel;
                    VF_TRY(dfd.upload(fds));
                    VF_TRY(dsel.upload(sel));
                    k_form_factors<<<(unsigned)fds.size(), 256, 0, st>>>(B.d_pd.p, dfd.p, dsel.p, B.Y.p, B.Z.p, B.small.p, buf->p);
                    VF_TRY_CUDA(cudaGetLastError());
                    VF_TRY_CUDA(cudaStreamSynchronize(st));
                    std::vector<uint8_t> ver_ok(fds.size(), 1);
                    if (o.verify) {
                        std::vector<double> ver_est;
                        VF_TRY(verify_factors(g, B, fds, buf->p, o.tol, o.seed ^ (uint64_t)h ^ ((uint64_t)attempt << 32),
                                              ver_ok, ver_est, st));
                    }
                    int32_t bi = (int32_t)stage_bufs.size();
                    std::vector<FactorDesc> fds2;
                    std::vector<int32_t> sel2, owner2;
                    int64_t fstage2 = 0;
                    for (size_t f = 0; f < fds.size(); ++f) {
                        int32_t id = fd_owner[f];
                        if (!ver_ok[f]) {
                            DNode& d = N[id];
                            const ProbeDesc& p = B.pd[fds[f].probe];
                            S.verify_failed++;
                            const int32_t q1 = fds[f].q + 1;
                            if (attempt < kVerifyRaise && q1 <= p.ell && q1 <= o.k_max &&
                                svd_bytes(q1, d.st.m1, d.st.n1) < d.best_alt) {
                                // one more rank from the same probe
                                FactorDesc g2 = fds[f];
                                g2.q = q1;
                                g2.sel_off = (int64_t)sel2.size();
                                for (int32_t k = 0; k < q1; ++k) sel2.push_back(orders[fds[f].probe][k]);
                                g2.u_off = fstage2;
                                fstage2 += (int64_t)(p.m1 + p.n1) * q1;
                                fds2.push_back(g2);
                                owner2.push_back(id);
                                d.q = q1;
                                continue;
                            }
                            // back to the rank doubling
                            d.q = 0;
                            const bool full = p.ell == std::min(p.m1, p.n1);
                            if (!full && 2 * d.k <= o.k_max && svd_bytes(d.k, d.st.m1, d.st.n1) < d.best_alt) {
                                d.k *= 2;
                                next.push_back(id);
                            } else {
                                S.probes_failed++;
                            }
                            continue;
                        }
                        stage_ref[id] = StageRef{bi, fds[f].u_off};
                        // keep the compacted lists of this candidate
                        const ProbeDesc& p = B.pd[fds[f].probe];
                        N[id].lists_off = (int64_t)lists_pool.size();
                        lists_pool.insert(lists_pool.end(), B.lists.begin() + p.rows_off,
                                          B.lists.begin() + p.rows_off + p.m1);
                        lists_pool.insert(lists_pool.end(), B.lists.begin() + p.cols_off,
                                          B.lists.begin() + p.cols_off + p.n1);
                    }
                    stage_bufs.push_back(std::move(buf));
                    fds.swap(fds2);
                    sel.swap(sel2);
                    fd_owner.swap(owner2);
                    fstage = fstage2;
                }
                pending.swap(next);
            }
            return VF_OK;
            };
            VF_TRY(probe_rounds(pending));
            // The audits: if the probes of audited skips won too often, the
            // predictor is off its training distribution at this level, and
            // the skipped candidates are probed after all.
            if (!audit.empty()) {
                int64_t wins = 0;
                for (int32_t id : audit) wins += (N[id].q > 0 && stage_ref[id].buf >= 0) ? 1 : 0;
                S.predictor_audits += (int64_t)audit.size();
                S.predictor_audit_wins += wins;
                if (wins >= 2 && wins * kAuditMaxWinInv > (int64_t)audit.size() && !skipped.empty()) {
                    S.predictor_fallbacks++;
                    S.probes_predicted_skip -= (int64_t)skipped.size();
                    for (int32_t id : skipped) N[id].k = std::min(o.k0, o.k_max);
                    log_ids.insert(log_ids.end(), skipped.begin(), skipped.end());
                    H->h_probe_feat.insert(H->h_probe_feat.end(), skipped_feat.begin(), skipped_feat.end());
                    VF_TRY(probe_rounds(skipped));
                }
            }
            // the probe log's labels: the rank bin of an accepted SVD, else "no SVD"
            for (size_t i = log0; i < log_ids.size(); ++i) {
                const DNode& d = N[log_ids[i]];
                int32_t c = VF_PRED_NCLASS - 1;
                if (d.q > 0 && stage_ref[log_ids[i]].buf >= 0) c = d.q <= 8 ? 0 : d.q <= 16 ? 1 : d.q <= 32 ? 2 : d.q <= 64 ? 3 : 4;
                H->h_probe_label.push_back(c);
            }
            // decisions for this level
            for (int32_t id : level) {
                DNode& d = N[id];
                if (h == 0 || d.kind == VF_BLK_ZERO) continue;
                int64_t mm = t->count[d.I], nn = t->count[d.J];
                int64_t bd = 4 * mm * nn, bc = csr_bytes(mm, d.st.nnz);
                // candidates in tie order: dense < CSR < SVD < hierarchical
                int32_t kind = VF_BLK_DENSE;
                int64_t best = bd;
                if (bc < best) { best = bc; kind = VF_BLK_CSR; }
                if (d.q > 0 && stage_ref[id].buf >= 0) {
                    int64_t bs = svd_bytes(d.q, d.st.m1, d.st.n1);
                    if (bs < best) { best = bs; kind = VF_BLK_SVD; }
                }
                if (d.hier_bytes < best) { best = d.hier_bytes; kind = VF_BLK_HIER; }
                if (kind == VF_BLK_HIER) {
                    bool all_csr = true, all_dense = true, any = false;
                    for (int32_t k = d.kid_begin; k < d.kid_end; ++k) {
                        int32_t kk = Bd.kid_kind(Bd.kids[k]);
                        if (kk == VF_BLK_ZERO) continue;
                        any = true;
                        all_csr = all_csr && kk == VF_BLK_CSR;
                        all_dense = all_dense && kk == VF_BLK_DENSE;
                    }
                    if (any && all_csr) { kind = VF_BLK_CSR; best = bc; }
                    else if (any && all_dense) { kind = VF_BLK_DENSE; best = bd; }
                }
                d.kind = kind;
                d.bytes = best;
            }
        }
        t3 = now_seconds();
        S.t_probe = t3 - t2;

        // ---------------- flatten to stored blocks
        std::vector<Kid> stack(Bd.top_refs.rbegin(), Bd.top_refs.rend());
        while (!stack.empty()) {
            Kid k = stack.back();
            stack.pop_back();
            HBlock b{};
            int32_t kind;
            if (k.ref >= 0) {
                const DNode& d = N[k.ref];
                kind = d.kind;
                if (kind == VF_BLK_HIER) {
                    S.nblocks[VF_BLK_HIER]++;
                    for (int32_t q = d.kid_end - 1; q >= d.kid_begin; --q) stack.push_back(Bd.kids[q]);
                    continue;
                }
                b.I = d.I;
                b.J = d.J;
                b.q = kind == VF_BLK_SVD ? d.q : 0;
                b.m1 = kind == VF_BLK_SVD ? d.st.m1 : (int32_t)d.st.nnz;
                b.n1 = kind == VF_BLK_SVD ? d.st.n1 : 0;
                hb_node.push_back(k.ref);
            } else {
                int64_t p = -1 - k.ref;
                int64_t a = p / Bd.nleaves, bb = p - a * Bd.nleaves;
                kind = Bd.leaf_pair_choice(p).first;
                // leaf node ids: find from leaf index via first position
                b.I = -1;
                b.J = -1;
                b.m1 = Bd.pnnz[p];
                b.r0 = Bd.leaf_first[a];
                b.m = Bd.leaf_count[a];
                b.c0 = Bd.leaf_first[bb];
                b.n = Bd.leaf_count[bb];
                hb_node.push_back(-1);
            }
            S.nblocks[kind]++;
            if (kind == VF_BLK_ZERO) { hb_node.pop_back(); continue; }
            b.kind = kind;
            if (b.I >= 0) {
                b.r0 = t->first[b.I];
                b.m = t->count[b.I];
                b.c0 = t->first[b.J];
                b.n = t->count[b.J];
            }
            HB.push_back(b);
        }
    }
    // resolve leaf-pair node ids (for vf_hmat_blocks)
    {
        std::vector<int32_t> node_of_first_leaf(n, -1);
        for (int32_t k = 0; k < nnodes; ++k)
            if (t->is_leaf(k)) node_of_first_leaf[t->first[k]] = k;
        for (auto& b : HB)
            if (b.I < 0) { b.I = node_of_first_leaf[b.r0]; b.J = node_of_first_leaf[b.c0]; }
    }
    // offsets
    int64_t nval = 0, naux = 0, nT = 0;
    int32_t maxq = 0;
    for (auto& b : HB) {
        b.off_val = nval;
        b.off_aux = naux;
        b.off_T = -1;
        if (b.kind == VF_BLK_DENSE) {
            nval += (int64_t)b.m * b.n;
            S.bytes[VF_BLK_DENSE] += 4ll * b.m * b.n;
        } else if (b.kind == VF_BLK_CSR) {
            nval += b.m1;
            naux += b.m + 1 + b.m1;
            S.bytes[VF_BLK_CSR] += 8ll * b.m1 + 4ll * (b.m + 1);
        } else {
            nval += (int64_t)(b.m1 + b.n1) * b.q;
            naux += b.m1 + b.n1;
            b.off_T = nT;
            nT += b.q;
            maxq = std::max(maxq, b.q);
            S.bytes[VF_BLK_SVD] += svd_bytes(b.q, b.m1, b.n1);
        }
        // keep values 16-byte aligned per block for vector loads
        nval = (nval + 3) & ~int64_t(3);
    }
    S.max_rank = maxq;
    H->n_val = nval;
    H->n_aux = naux;
    H->n_T = nT;
    H->max_q = maxq;
    // pools are padded by 16 elements: the multiply copies 16-byte aligned supersets
    VF_TRY(H->val.alloc(nval + 16));
    VF_TRY(H->aux.alloc(naux + 16));
    VF_TRY_CUDA(cudaMemsetAsync(H->val.p, 0, (nval + 16) * 4, st));
    VF_TRY_CUDA(cudaMemsetAsync(H->aux.p, 0, (naux + 16) * 4, st));
    // pack
    std::vector<PackDesc> pk_dense, pk_csr;
    std::vector<std::vector<PackDesc>> pk_svd(stage_bufs.size());
    dbuf<int32_t> dlists;
    VF_TRY(dlists.upload(lists_pool));
    for (size_t bi = 0; bi < HB.size(); ++bi) {
        const HBlock& b = HB[bi];
        PackDesc p{};
        p.kind = b.kind;
        p.r0 = b.r0;
        p.m = b.m;
        p.c0 = b.c0;
        p.n = b.n;
        p.off_val = b.off_val;
        p.off_aux = b.off_aux;
        p.q = b.q;
        p.m1 = b.m1;
        p.n1 = b.n1;
        if (b.kind == VF_BLK_DENSE) pk_dense.push_back(p);
        else if (b.kind == VF_BLK_CSR) pk_csr.push_back(p);
        else {
            int32_t id = hb_node[bi];
            p.stage_off = stage_ref[id].off;
            p.lists_off = N[id].lists_off;
            pk_svd[stage_ref[id].buf].push_back(p);
        }
    }
    // row tiles of the multiply: runs of consecutive leaves holding <= 64 rows
    H->h_tile_first.clear();
    H->h_tile_count.clear();
    for (size_t k = 0; k < Bd.leaf_first.size(); ++k) {
        if (!H->h_tile_first.empty() && H->h_tile_count.back() + Bd.leaf_count[k] <= 64) {
            H->h_tile_count.back() += Bd.leaf_count[k];
        } else {
            H->h_tile_first.push_back(Bd.leaf_first[k]);
            H->h_tile_count.push_back(Bd.leaf_count[k]);
        }
    }
    if (!pk_dense.empty()) {
        dbuf<PackDesc> d;
        dbuf<int32_t> d_tor, d_tf, d_tc;
        std::vector<int32_t> tor(n);
        for (size_t k = 0; k < H->h_tile_first.size(); ++k)
            for (int32_t r = H->h_tile_first[k]; r < H->h_tile_first[k] + H->h_tile_count[k]; ++r) tor[r] = (int32_t)k;
        VF_TRY(d_tor.upload(tor));
        VF_TRY(d_tf.upload(H->h_tile_first));
        VF_TRY(d_tc.upload(H->h_tile_count));
        VF_TRY(d.upload(pk_dense));
        k_pack_dense<<<(unsigned)pk_dense.size(), 256, 0, st>>>(g, d.p, d_tor.p, d_tf.p, d_tc.p, H->val.p);
        VF_TRY_CUDA(cudaGetLastError());
        VF_TRY_CUDA(cudaStreamSynchronize(st));
    }
    if (!pk_csr.empty()) {
        dbuf<PackDesc> d;
        VF_TRY(d.upload(pk_csr));
        k_pack_csr<<<(unsigned)pk_csr.size(), 256, 0, st>>>(g, d.p, H->val.p, H->aux.p);
        VF_TRY_CUDA(cudaGetLastError());
        VF_TRY_CUDA(cudaStreamSynchronize(st));
    }
    for (size_t bi = 0; bi < pk_svd.size(); ++bi) {
        if (pk_svd[bi].empty()) continue;
        dbuf<PackDesc> d;
        VF_TRY(d.upload(pk_svd[bi]));
        k_pack_svd<<<(unsigned)pk_svd[bi].size(), 256, 0, st>>>(d.p, dlists.p, stage_bufs[bi]->p, H->val.p, H->aux.p);
        VF_TRY_CUDA(cudaGetLastError());
        VF_TRY_CUDA(cudaStreamSynchronize(st));
    }
    stage_bufs.clear();
    VF_TRY(H->blocks.upload(HB));
    // low-precision copies
    if (o.precisions & (1u << VF_PREC_BF16)) {
        VF_TRY(H->val16.alloc(nval + 16));
        k_to_bf16<<<1024, 256, 0, st>>>(H->val.p, H->val16.p, nval + 16);
        VF_TRY_CUDA(cudaGetLastError());
        H->has_bf16 = true;
    }
    if (o.precisions & (1u << VF_PREC_FP8)) {
        VF_TRY(H->val8.alloc(nval + 16));
        VF_TRY(H->scale8.alloc(std::max<size_t>(HB.size(), 1)));
        VF_TRY_CUDA(cudaMemsetAsync(H->val8.p, 0, nval + 16, st));
        if (!HB.empty()) k_to_fp8<<<(unsigned)HB.size(), 256, 0, st>>>(H->blocks.p, H->val.p, H->val8.p, H->scale8.p);
        VF_TRY_CUDA(cudaGetLastError());
        H->has_fp8 = true;
    }
    VF_TRY_CUDA(cudaStreamSynchronize(st));
    double t4 = now_seconds();
    S.t_pack = t4 - t3;
    // ---------------- the multiply's pages over the row tiles
    VF_TRY(H->upload_all());
    S.t_total = now_seconds() - t0;
    H->stats = S;
    if (stats_out) *stats_out = S;
    *out = H.release();
    return VF_OK;
}

extern "C" vf_status vf_hmat_probe_log(const vf_hmat* h, int64_t* n, float* feats, int32_t* labels) {
    clear_error();
    VF_CHECK(h && n, VF_E_INVAL, "vf_hmat_probe_log: null argument");
    *n = (int64_t)h->h_probe_label.size();
    if (feats) std::copy(h->h_probe_feat.begin(), h->h_probe_feat.end(), feats);
    if (labels) std::copy(h->h_probe_label.begin(), h->h_probe_label.end(), labels);
    return VF_OK;
}
