// Thermal quantities built on the compressed multiply and the Jacobi solve:
// the equilibrium temperatures of Section 5.1 (two radiosity systems and the
// surface energy balance, Eq. 3d-equilbr) and the flux updates of
// Algorithm 6 (Section 5.2), whose two multiplies by F run as one multiply
// of 2R right-hand sides.
//
// Layout: every vector is face order, column-major N x R with an explicit
// leading dimension.  Temporaries are stream-ordered allocations
// (cudaMallocAsync) released on the caller's stream.
#include <cmath>

#include "vf_internal.cuh"

namespace vf {

constexpr double kSigmaSB = 5.670374419e-8;  // CODATA 2018 (W m^-2 K^-4)

// A stream-ordered device buffer (released on its stream).
struct sbuf {
    float* p = nullptr;
    cudaStream_t st = nullptr;
    explicit sbuf(cudaStream_t s) : st(s) {}
    sbuf(const sbuf&) = delete;
    sbuf& operator=(const sbuf&) = delete;
    ~sbuf() {
        if (p) cudaFreeAsync(p, st);
    }
    vf_status alloc(size_t floats) {
        cudaError_t e = inject_alloc_failure() ? cudaErrorMemoryAllocation
                                               : cudaMallocAsync((void**)&p, floats * sizeof(float), st);
        if (e != cudaSuccess) {
            p = nullptr;
            set_error("device allocation of %zu bytes failed: %s", floats * sizeof(float), cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? VF_E_NOMEM : VF_E_CUDA;
        }
        return VF_OK;
    }
};

__device__ __forceinline__ float pick(const float* v, float u, int64_t i) { return v ? v[i] : u; }

// out = a .* Q (ld_out = n)
__global__ void k_scale_cols(const float* __restrict__ Q, int64_t ldq, const float* __restrict__ a, float a_u,
                             int64_t n, int R, float* __restrict__ out) {
    const int64_t tot = n * (int64_t)R;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, i = e - c * n;
        out[e] = pick(a, a_u, i) * Q[c * ldq + i];
    }
}

// Qvis = Qdir + FW (Section 5.1: Q_direct + Q_refl), rhs = (1 - albedo) Qvis + H
__global__ void k_vis_and_ir_rhs(const float* __restrict__ Qdir, int64_t lde, const float* __restrict__ FW,
                                 const float* __restrict__ alb, float alb_u, const float* __restrict__ H, int64_t n,
                                 int R, float* __restrict__ Qvis, int64_t ldv, float* __restrict__ rhs) {
    const int64_t tot = n * (int64_t)R;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, i = e - c * n;
        const float v = Qdir[c * lde + i] + FW[e];
        Qvis[c * ldv + i] = v;
        rhs[e] = (1.f - pick(alb, alb_u, i)) * v + (H ? H[i] : 0.f);
    }
}

// Eq. 3d-equilbr: eps sigma T^4 = (1 - albedo) Qvis + eps Qir (FP64, clamped at 0)
__global__ void k_temperature(const float* __restrict__ Qvis, int64_t ldv, const float* __restrict__ Qir,
                              int64_t ldi, const float* __restrict__ alb, float alb_u, const float* __restrict__ eps,
                              float eps_u, int64_t n, int R, float* __restrict__ T, int64_t ldt) {
    const int64_t tot = n * (int64_t)R;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, i = e - c * n;
        const double a = pick(alb, alb_u, i), ep = pick(eps, eps_u, i);
        const double q = (1.0 - a) * (double)Qvis[c * ldv + i] + ep * (double)Qir[c * ldi + i];
        T[c * ldt + i] = (float)sqrt(sqrt(fmax(q, 0.0) / (ep * kSigmaSB)));
    }
}

// Algorithm 6 inputs of the two multiplies, as one N x 2R block:
// X[:, c] = albedo .* (Qdir' + Qrefl), X[:, R + c] = Qrad + (1 - eps) .* Qir
__global__ void k_step_in(const float* __restrict__ Qdir, const float* __restrict__ Qrefl,
                          const float* __restrict__ Qir, const float* __restrict__ Qrad, int64_t ld,
                          const float* __restrict__ alb, float alb_u, const float* __restrict__ eps, float eps_u,
                          int64_t n, int R, float* __restrict__ X) {
    const int64_t tot = n * (int64_t)R;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, i = e - c * n, o = c * ld + i;
        X[e] = pick(alb, alb_u, i) * (Qdir[o] + Qrefl[o]);
        X[tot + e] = Qrad[o] + (1.f - pick(eps, eps_u, i)) * Qir[o];
    }
}

// Qrefl' = Y[:, c], Qir' = Y[:, R + c], Qabs' = (1 - albedo)(Qdir' + Qrefl') + eps Qir'
__global__ void k_step_out(const float* __restrict__ Y, const float* __restrict__ Qdir, int64_t ld,
                           const float* __restrict__ alb, float alb_u, const float* __restrict__ eps, float eps_u,
                           int64_t n, int R, float* __restrict__ Qrefl, float* __restrict__ Qir,
                           float* __restrict__ Qabs) {
    const int64_t tot = n * (int64_t)R;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, i = e - c * n, o = c * ld + i;
        const float qr = Y[e], qi = Y[tot + e];
        Qrefl[o] = qr;
        Qir[o] = qi;
        Qabs[o] = (1.f - pick(alb, alb_u, i)) * (Qdir[o] + qr) + pick(eps, eps_u, i) * qi;
    }
}

static unsigned grid_for(int64_t tot) { return (unsigned)std::min<int64_t>(ceil_div(tot, 256), 4096); }

}  // namespace vf

using namespace vf;

extern "C" vf_status vf_equilibrium(const vf_hmat* h, const float* E, int64_t lde, int32_t R, const float* albedo,
                                    const float* emissivity, const float* H, const vf_equilibrium_opts* opts_in,
                                    float* Qvis, float* Qir, float* T, int64_t ld, vf_solve_stats* stats,
                                    vf_stream stream) {
    clear_error();
    VF_CHECK(h && E && T && opts_in, VF_E_INVAL, "vf_equilibrium: null argument");
    const int64_t n = vf_hmat_nfacets(h);
    VF_CHECK(R >= 1 && lde >= n && ld >= n, VF_E_INVAL, "vf_equilibrium: need R >= 1 and ld >= N");
    const vf_equilibrium_opts& o = *opts_in;
    VF_CHECK(albedo || (o.albedo >= 0.f && o.albedo < 1.f), VF_E_INVAL, "vf_equilibrium: albedo must be in [0, 1)");
    VF_CHECK(emissivity || (o.emissivity > 0.f && o.emissivity <= 1.f), VF_E_INVAL,
             "vf_equilibrium: emissivity must be in (0, 1]");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nR = (size_t)n * R;
    sbuf W(st), FW(st), rhs(st), vis(st), ir(st);
    VF_TRY(W.alloc(nR));
    VF_TRY(FW.alloc(nR));
    VF_TRY(rhs.alloc(nR));
    float* qv = Qvis;
    float* qi = Qir;
    int64_t ldv = ld, ldi = ld;
    if (!qv) {
        VF_TRY(vis.alloc(nR));
        qv = vis.p;
        ldv = n;
    }
    if (!qi) {
        VF_TRY(ir.alloc(nR));
        qi = ir.p;
        ldi = n;
    }
    vf_solve_opts so{};
    so.rtol = o.rtol > 0 ? o.rtol : 1e-6;
    so.max_iter = o.max_iter > 0 ? o.max_iter : 200;
    so.precision = o.precision;
    so.refine = o.refine;
    so.max_refine = 8;
    so.inner_rtol = 1e-3;
    so.clamp = 0;
    // Eq. time-indep-system-1 with W = diag(albedo) Q_vis: W = diag(albedo) Q_direct
    // + diag(albedo) F W, a radiosity system with rho = albedo; then
    // Q_vis = Q_direct + F W (Q_refl = F diag(albedo) Q_vis)
    k_scale_cols<<<grid_for((int64_t)nR), 256, 0, st>>>(E, lde, albedo, o.albedo, n, R, rhs.p);
    VF_TRY_CUDA(cudaGetLastError());
    so.rho = o.albedo;
    vf_solve_stats s1{}, s2{};
    vf_status r1 = vf_solve(h, albedo, rhs.p, n, W.p, n, R, &so, &s1, stream);
    if (r1 != VF_OK && r1 != VF_E_NOCONV) return r1;
    VF_TRY(vf_apply(h, (vf_precision)(o.refine ? VF_PREC_FP32 : o.precision), W.p, n, R, FW.p, n, stream));
    k_vis_and_ir_rhs<<<grid_for((int64_t)nR), 256, 0, st>>>(E, lde, FW.p, albedo, o.albedo, H, n, R, qv, ldv,
                                                             rhs.p);
    VF_TRY_CUDA(cudaGetLastError());
    // Eq. time-indep-system-2: (I - F) Q_IR = F ((1 - albedo) Q_vis + H), i.e.
    // Q_IR = F rhs + F Q_IR, a radiosity system with rho = 1 and E = F rhs
    VF_TRY(vf_apply(h, (vf_precision)(o.refine ? VF_PREC_FP32 : o.precision), rhs.p, n, R, FW.p, n, stream));
    so.rho = 1.f;
    vf_status r2 = vf_solve(h, nullptr, FW.p, n, qi, ldi, R, &so, &s2, stream);
    if (r2 != VF_OK && r2 != VF_E_NOCONV) return r2;
    k_temperature<<<grid_for((int64_t)nR), 256, 0, st>>>(qv, ldv, qi, ldi, albedo, o.albedo, emissivity,
                                                          o.emissivity, n, R, T, ld);
    VF_TRY_CUDA(cudaGetLastError());
    if (stats) {
        stats[0] = s1;
        stats[1] = s2;
    }
    VF_TRY_CUDA(cudaStreamSynchronize(st));
    if (r1 == VF_E_NOCONV || r2 == VF_E_NOCONV) {
        set_error("vf_equilibrium: a solve did not converge (Q_vis %d, Q_IR %d)", (int)s1.converged,
                  (int)s2.converged);
        return VF_E_NOCONV;
    }
    return VF_OK;
}

extern "C" vf_status vf_flux_step(const vf_hmat* h, vf_precision p, int32_t R, const float* albedo,
                                  const float* emissivity, float albedo_u, float emissivity_u,
                                  const float* Edirect_next, float* Qrefl, float* Qir, const float* Qrad, float* Qabs,
                                  int64_t ld, vf_stream stream) {
    clear_error();
    VF_CHECK(h && Edirect_next && Qrefl && Qir && Qrad && Qabs, VF_E_INVAL, "vf_flux_step: null argument");
    const int64_t n = vf_hmat_nfacets(h);
    VF_CHECK(R >= 1 && ld >= n, VF_E_INVAL, "vf_flux_step: need R >= 1 and ld >= N");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nR = (size_t)n * R;
    sbuf X(st), Y(st);
    VF_TRY(X.alloc(2 * nR));
    VF_TRY(Y.alloc(2 * nR));
    k_step_in<<<grid_for((int64_t)nR), 256, 0, st>>>(Edirect_next, Qrefl, Qir, Qrad, ld, albedo, albedo_u,
                                                      emissivity, emissivity_u, n, R, X.p);
    VF_TRY_CUDA(cudaGetLastError());
    // both fluxes' multiplies as one multiply of 2R right-hand sides
    VF_TRY(vf_apply(h, p, X.p, n, 2 * R, Y.p, n, stream));
    k_step_out<<<grid_for((int64_t)nR), 256, 0, st>>>(Y.p, Edirect_next, ld, albedo, albedo_u, emissivity,
                                                       emissivity_u, n, R, Qrefl, Qir, Qabs);
    VF_TRY_CUDA(cudaGetLastError());
    return VF_OK;
}
