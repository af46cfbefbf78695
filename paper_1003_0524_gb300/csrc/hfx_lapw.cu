// hfx_lapw.cu -- the exchange matrix in the LAPW basis of every k
// (Eq. APW trafo, Sec. III.A), the step after the build:
//
//   V_GG'(k) = sum_{n,n'} (S c)[G][n] V^x[n][n'] (c^H S)[n'][G'] = B^H (V^x B),
//   B = c^H S  (n_bands x npw),
//
// with S_GG'(k) = <chi_G|chi_G'> the overlap of the basis functions of k and c
// the band coefficients given to hfx_set_kpoint.  Three batched complex FP64
// GEMMs over all k (B, then W = V^x B, then B^H W): a few tens of GFLOP per SCF
// step, well under a percent of the build, so they run on the FP64 units.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "hfx_internal.cuh"

using namespace hfx;

namespace {

bool finite_all(const double *p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

}  // namespace

extern "C" {

int hfx_set_overlap(hfx_ctx *ctx, int ik, const double *S, int ld) {
    if (!ctx) return HFX_EINVAL;
    if (ik < 0 || ik >= ctx->nk || !S) return set_err(ctx, HFX_EINVAL, "set_overlap: bad k or pointer");
    KPoint &k = ctx->kp[ik];
    if (!k.set) return set_err(ctx, HFX_EMISSING, "set_overlap: set_kpoint(k) comes first");
    const int n = k.npw;
    if (ld < n) return set_err(ctx, HFX_EINVAL, "set_overlap: leading dimension below npw");
    std::vector<double> Sc(2 * (size_t)n * n);
    for (int i = 0; i < n; ++i) std::memcpy(Sc.data() + 2 * (size_t)i * n, S + 2 * (size_t)i * ld, 16 * (size_t)n);
    if (!finite_all(Sc.data(), Sc.size())) return set_err(ctx, HFX_ENONFINITE, "set_overlap: non-finite element");
    double mx = 0.0, dev = 0.0;
    for (size_t i = 0; i < Sc.size(); ++i) mx = std::max(mx, std::fabs(Sc[i]));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            const double *a = Sc.data() + 2 * ((size_t)i * n + j), *b = Sc.data() + 2 * ((size_t)j * n + i);
            dev = std::max(dev, std::fabs(a[0] - b[0]) + std::fabs(a[1] + b[1]));
        }
    if (dev > ctx->opt.herm_tol * std::max(mx, 1e-300)) return set_err(ctx, HFX_ENOTHERM, "set_overlap: S is not Hermitian");
    if (ctx->S_npw.size() != (size_t)ctx->nk) { ctx->S_npw.assign(ctx->nk, 0); ctx->d_S.assign(ctx->nk, nullptr); }
    int rc = cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
    if (rc) return rc;
    if (ctx->S_npw[ik] != n) {
        if (ctx->d_S[ik]) cudaFree(ctx->d_S[ik]);
        ctx->d_S[ik] = nullptr;
        ctx->S_npw[ik] = 0;
        if ((rc = cuda_check(ctx, cudaMalloc(&ctx->d_S[ik], sizeof(double2) * std::max<size_t>(1, (size_t)n * n)),
                             "overlap buffer")))
            return rc;
        ctx->S_npw[ik] = n;
    }
    return cuda_check(ctx, cudaMemcpy(ctx->d_S[ik], Sc.data(), 16 * (size_t)n * n, cudaMemcpyHostToDevice), "copy S");
}

int hfx_lapw_transform_all(hfx_ctx *ctx, hfx_stats *st) {
    if (!ctx) return HFX_EINVAL;
    if (!ctx->built) return set_err(ctx, HFX_EMISSING, "lapw_transform_all: no complete build");
    const int nk = ctx->nk;
    for (int ik = 0; ik < nk; ++ik)
        if (ctx->S_npw.size() != (size_t)nk || ctx->S_npw[ik] != ctx->kp[ik].npw)
            return set_err(ctx, HFX_EMISSING, "lapw_transform_all: set_overlap missing for k " + std::to_string(ik));
    int rc = cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
    if (rc) return rc;
    // buffers: per k, B and W (nb x npw) and V_GG' (npw x npw)
    std::vector<size_t> oB(nk), oW(nk), oV(nk);
    size_t tot = 0;
    for (int ik = 0; ik < nk; ++ik) {
        const size_t nb = ctx->kp[ik].nb, np = ctx->kp[ik].npw;
        oB[ik] = tot; tot += nb * np;
        oW[ik] = tot; tot += nb * np;
        oV[ik] = tot; tot += np * np;
    }
    if ((rc = scratch_reserve(ctx, ctx->s_lapw, tot * sizeof(double2)))) return rc;
    double2 *base = reinterpret_cast<double2 *>(ctx->s_lapw.p);
    std::vector<ZGemmBatch> g1(nk), g2(nk), g3(nk);
    int maxnp = 0, maxnb = 0;
    double flops = 0.0;
    for (int ik = 0; ik < nk; ++ik) {
        const KPoint &k = ctx->kp[ik];
        const int nb = k.nb, np = k.npw;
        maxnp = std::max(maxnp, np);
        maxnb = std::max(maxnb, nb);
        double2 *B = base + oB[ik], *W = base + oW[ik], *Vg = base + oV[ik];
        // B[n][G'] = sum_G'' conj(c[n][G'']) S[G''][G']
        ZGemmBatch &a = g1[ik];
        a.A = k.d_c; a.B = ctx->d_S[ik]; a.C = B;
        a.M = nb; a.N = np; a.K1 = 1; a.K2 = np;
        a.sAi = np; a.sAk1 = 0; a.sAk2 = 1; a.sBk1 = 0; a.sBk2 = np; a.sBj = 1; a.sCi = np; a.sCj = 1; a.conjA = 1;
        // W[n][G'] = sum_n' V[n][n'] B[n'][G']
        ZGemmBatch &b = g2[ik];
        b.A = ctx->d_V[ik]; b.B = B; b.C = W;
        b.M = nb; b.N = np; b.K1 = 1; b.K2 = nb;
        b.sAi = nb; b.sAk1 = 0; b.sAk2 = 1; b.sBk1 = 0; b.sBk2 = np; b.sBj = 1; b.sCi = np; b.sCj = 1; b.conjA = 0;
        // V_GG'[G][G'] = sum_n conj(B[n][G]) W[n][G']
        ZGemmBatch &d = g3[ik];
        d.A = B; d.B = W; d.C = Vg;
        d.M = np; d.N = np; d.K1 = 1; d.K2 = nb;
        d.sAi = 1; d.sAk1 = 0; d.sAk2 = np; d.sBk1 = 0; d.sBk2 = np; d.sBj = 1; d.sCi = np; d.sCj = 1; d.conjA = 1;
        flops += 8.0 * ((double)nb * np * np + (double)nb * nb * np + (double)np * np * nb);
    }
    if ((rc = scratch_reserve(ctx, ctx->s_lapw_tab, 3 * (size_t)nk * sizeof(ZGemmBatch)))) return rc;
    ZGemmBatch *dt = reinterpret_cast<ZGemmBatch *>(ctx->s_lapw_tab.p);
    std::vector<ZGemmBatch> all(g1);
    all.insert(all.end(), g2.begin(), g2.end());
    all.insert(all.end(), g3.begin(), g3.end());
    if ((rc = cuda_check(ctx, cudaMemcpyAsync(dt, all.data(), all.size() * sizeof(ZGemmBatch), cudaMemcpyHostToDevice,
                                              ctx->stream),
                         "lapw tables")))
        return rc;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, ctx->stream);
    launch_zgemm64(dt, nk, maxnb, maxnp, ctx->stream);
    launch_zgemm64(dt + nk, nk, maxnb, maxnp, ctx->stream);
    launch_zgemm64(dt + 2 * nk, nk, maxnp, maxnp, ctx->stream);
    cudaEventRecord(e1, ctx->stream);
    rc = cuda_check(ctx, cudaGetLastError(), "lapw transform");
    if (!rc) rc = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "stream synchronize");
    if (!rc && st) {
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        std::memset(st, 0, sizeof(*st));
        st->ms_total = t;
        st->useful_flops = flops;
        st->n_launches = 3;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    ctx->lapw_off = oV;
    ctx->lapw_valid = true;
    return HFX_OK;
}

int hfx_get_lapw_exchange(hfx_ctx *ctx, int ik, double *Vgg, int ld) {
    if (!ctx) return HFX_EINVAL;
    if (ik < 0 || ik >= ctx->nk || !Vgg) return set_err(ctx, HFX_EINVAL, "get_lapw_exchange: bad k or pointer");
    if (!ctx->lapw_valid || !ctx->built) return set_err(ctx, HFX_EMISSING, "get_lapw_exchange: no transform of the last build");
    const int np = ctx->kp[ik].npw;
    if (ld < np) return set_err(ctx, HFX_EINVAL, "get_lapw_exchange: leading dimension below npw");
    const double2 *src = reinterpret_cast<const double2 *>(ctx->s_lapw.p) + ctx->lapw_off[ik];
    return cuda_check(ctx, cudaMemcpy2D(Vgg, 16 * (size_t)ld, src, 16 * (size_t)np, 16 * (size_t)np, np, cudaMemcpyDeviceToHost),
                      "copy V_GG'");
}

}  // extern "C"
