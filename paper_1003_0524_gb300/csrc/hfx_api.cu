// hfx_api.cu -- C ABI of the exchange-matrix library: input validation,
// device-resident inputs, q batching and the two build pipelines
// (FP64, and BF16x3 split products on the tensor cores).
#include <type_traits>
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hfx_internal.cuh"

namespace hfx {

int set_err(hfx_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

int cuda_check(hfx_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return HFX_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_err(ctx, HFX_ENOMEM, std::string(what) + ": " + cudaGetErrorString(e));
    }
    return set_err(ctx, HFX_EDEVICE, std::string(what) + ": " + cudaGetErrorString(e));
}

int scratch_reserve(hfx_ctx *ctx, Scratch &s, size_t bytes) {
    if (bytes <= s.bytes) return HFX_OK;
    if (s.p) cudaFree(s.p);
    s.p = nullptr;
    s.bytes = 0;
    size_t b = std::max<size_t>(bytes, 256);
    int rc = cuda_check(ctx, cudaMalloc(&s.p, b), "device allocation");
    if (rc) return rc;
    s.bytes = b;
    return HFX_OK;
}

}  // namespace hfx

using namespace hfx;

namespace {

template <typename T> int dalloc(hfx_ctx *ctx, T **p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    return cuda_check(ctx, cudaMalloc((void **)p, n * sizeof(T)), "device allocation");
}

void dfree(void *p) {
    if (p) cudaFree(p);
}

template <typename T> int h2d(hfx_ctx *ctx, T *dst, const T *src, size_t n) {
    if (n == 0) return HFX_OK;
    return cuda_check(ctx, cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyHostToDevice, ctx->stream), "copy to device");
}

bool finite_all(const double *p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

long long rup(long long x, long long m) { return (x + m - 1) / m * m; }

int sync(hfx_ctx *ctx) { return cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "stream synchronize"); }

int check_dev_err(hfx_ctx *ctx) {
    int e = 0;
    int rc = cuda_check(ctx, cudaMemcpy(&e, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost), "error word");
    if (rc) return rc;
    if (e) {
        int z = 0;
        cudaMemcpy(ctx->d_err, &z, sizeof(int), cudaMemcpyHostToDevice);
        return set_err(ctx, e == kDevBadIndex ? HFX_EDEVICE : HFX_ETIMEOUT,
                       "device wait expired or bad index in a kernel (code " + std::to_string(e) + ")");
    }
    return HFX_OK;
}

struct Batch {
    std::vector<int> qs;            // global q indices
    std::vector<QDesc> qd;
    std::vector<PairDesc> pairs;
    long long ncols = 0;
};

}  // namespace

extern "C" {

void hfx_default_options(hfx_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = HFX_PREC_SLICED;
    opt->sparse = HFX_SPARSE_AUTO;
    opt->q0_term = 1;
    opt->beta = 0.005;
    opt->herm_tol = 1e-10;
    opt->sparse_tol = 1e-12;
    opt->stream = nullptr;
    opt->device = 0;
    opt->work_bytes = 0;
}

const char *hfx_strerror(int code) {
    switch (code) {
    case HFX_OK: return "ok";
    case HFX_EINVAL: return "invalid argument";
    case HFX_ENOTHERM: return "Coulomb matrix is not Hermitian";
    case HFX_ENONFINITE: return "non-finite input";
    case HFX_EMISSING: return "missing input (set_radial / set_kpoint / set_coulomb)";
    case HFX_EDEVICE: return "CUDA error";
    case HFX_ETIMEOUT: return "bounded device wait expired";
    case HFX_ENOMEM: return "out of memory";
    case HFX_ENOTSPARSE: return "Coulomb matrix is not block-sparse after the multipole transform";
    case HFX_EUNSUPPORTED: return "unsupported size or option";
    default: return "unknown status";
    }
}

const char *hfx_last_error(const hfx_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

const char *hfx_version(void) { return "hfx-gb300 0.1 (sm_103a)"; }

int hfx_create(const hfx_system *sys, const hfx_options *opt_in, hfx_ctx **out) {
    if (!out) return HFX_EINVAL;
    *out = nullptr;
    if (!sys || !sys->pos_frac || !sys->rmt) return HFX_EINVAL;
    if (sys->n_atoms < 1 || sys->n_atoms > kMaxAtoms) return HFX_EINVAL;
    if (sys->lmax < 0 || sys->lmax > kMaxL || sys->Lmax < 0 || sys->Lmax > kMaxL) return HFX_EINVAL;
    if (sys->n_rad < 1 || sys->n_rad > kMaxP) return HFX_EINVAL;
    for (int i = 0; i < 3; ++i)
        if (sys->mesh[i] < 1 || sys->mesh[i] > 64) return HFX_EINVAL;
    if (!finite_all(sys->lattice, 9) || !finite_all(sys->pos_frac, 3 * (size_t)sys->n_atoms) ||
        !finite_all(sys->rmt, sys->n_atoms))
        return HFX_ENONFINITE;
    hfx_options opt;
    if (opt_in) opt = *opt_in;
    else hfx_default_options(&opt);
    if (opt.precision != HFX_PREC_FP64 && opt.precision != HFX_PREC_SLICED) return HFX_EINVAL;
    if (opt.sparse < 0 || opt.sparse > 2 || !(opt.beta > 0.0 && opt.beta < 1.0)) return HFX_EINVAL;

    hfx_ctx *ctx = new (std::nothrow) hfx_ctx();
    if (!ctx) return HFX_ENOMEM;
    ctx->sys = *sys;
    ctx->opt = opt;
    ctx->pos.assign(sys->pos_frac, sys->pos_frac + 3 * sys->n_atoms);
    ctx->rmt.assign(sys->rmt, sys->rmt + sys->n_atoms);
    ctx->sys.pos_frac = ctx->pos.data();
    ctx->sys.rmt = ctx->rmt.data();
    const double *a = sys->lattice;
    double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) + a[2] * (a[3] * a[7] - a[4] * a[6]);
    if (!(std::fabs(det) > 1e-9)) { delete ctx; return HFX_EINVAL; }
    ctx->omega = std::fabs(det);
    // B = 2 pi A^{-T}
    double inv[9];
    inv[0] = (a[4] * a[8] - a[5] * a[7]) / det; inv[1] = (a[2] * a[7] - a[1] * a[8]) / det; inv[2] = (a[1] * a[5] - a[2] * a[4]) / det;
    inv[3] = (a[5] * a[6] - a[3] * a[8]) / det; inv[4] = (a[0] * a[8] - a[2] * a[6]) / det; inv[5] = (a[2] * a[3] - a[0] * a[5]) / det;
    inv[6] = (a[3] * a[7] - a[4] * a[6]) / det; inv[7] = (a[1] * a[6] - a[0] * a[7]) / det; inv[8] = (a[0] * a[4] - a[1] * a[3]) / det;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) ctx->B[3 * i + j] = 2.0 * M_PI * inv[3 * j + i];
    // spheres must not overlap (within one cell and with the nearest images)
    for (int i = 0; i < sys->n_atoms; ++i) {
        if (sys->rmt[i] < 0.0) { delete ctx; return HFX_EINVAL; }
        for (int j = 0; j < sys->n_atoms; ++j)
            for (int t0 = -1; t0 <= 1; ++t0)
                for (int t1 = -1; t1 <= 1; ++t1)
                    for (int t2 = -1; t2 <= 1; ++t2) {
                        if (i == j && !t0 && !t1 && !t2) continue;
                        double f[3] = {sys->pos_frac[3 * j] - sys->pos_frac[3 * i] + t0,
                                       sys->pos_frac[3 * j + 1] - sys->pos_frac[3 * i + 1] + t1,
                                       sys->pos_frac[3 * j + 2] - sys->pos_frac[3 * i + 2] + t2};
                        double c[3] = {0, 0, 0};
                        for (int x = 0; x < 3; ++x) c[x] = f[0] * a[x] + f[1] * a[3 + x] + f[2] * a[6 + x];
                        double d = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
                        if (d < sys->rmt[i] + sys->rmt[j] - 1e-12) {
                            delete ctx;
                            return HFX_EINVAL;
                        }
                    }
    }
    ctx->nk = sys->mesh[0] * sys->mesh[1] * sys->mesh[2];
    ctx->nlm = (sys->lmax + 1) * (sys->lmax + 1);
    ctx->nLM = (sys->Lmax + 1) * (sys->Lmax + 1);
    ctx->nlmp = 2 * ctx->nlm;
    ctx->nlp = 2 * (sys->lmax + 1);
    ctx->P = sys->n_rad;
    ctx->nch = sys->n_atoms * ctx->nLM;
    ctx->nmt = ctx->nch * ctx->P;
    ctx->kp.resize(ctx->nk);
    ctx->qp.resize(ctx->nk);
    ctx->rset.assign(sys->n_atoms, 0);
    ctx->d_V.assign(ctx->nk, nullptr);
    ctx->device = opt.device;
    int rc = cuda_check(ctx, cudaSetDevice(opt.device), "cudaSetDevice");
    if (rc) { delete ctx; return rc; }
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, opt.device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, opt.device);
    if (major != 10) {
        set_err(ctx, HFX_EUNSUPPORTED, "this library is built for sm_103a (GB300)");
        rc = HFX_EUNSUPPORTED;
        delete ctx;
        return rc;
    }
    ctx->stream = reinterpret_cast<cudaStream_t>(opt.stream);
    size_t nR = (size_t)sys->n_atoms * (sys->Lmax + 1) * ctx->P * ctx->nlp * ctx->nlp;
    if ((rc = dalloc(ctx, &ctx->d_R, nR)) || (rc = dalloc(ctx, &ctx->d_mu, (size_t)sys->n_atoms * (sys->Lmax + 1) * ctx->P)) ||
        (rc = dalloc(ctx, &ctx->d_T, (size_t)sys->n_atoms * (sys->Lmax + 1) * ctx->P * ctx->P)) ||
        (rc = dalloc(ctx, &ctx->d_gaunt, (size_t)ctx->nLM * ctx->nlm * (sys->lmax + 1))) ||
        (rc = dalloc(ctx, &ctx->d_posf, (size_t)3 * sys->n_atoms + sys->n_atoms)) ||
        (rc = dalloc(ctx, &ctx->d_err, 1)) || (rc = dalloc(ctx, &ctx->d_Ex, 1))) {
        hfx_destroy(ctx);
        return rc;
    }
    cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream);
    std::vector<double> pr(ctx->pos);
    pr.insert(pr.end(), ctx->rmt.begin(), ctx->rmt.end());
    if ((rc = h2d(ctx, ctx->d_posf, pr.data(), pr.size()))) { hfx_destroy(ctx); return rc; }
    launch_gaunt(ctx->d_gaunt, sys->Lmax, sys->lmax, ctx->stream);
    if ((rc = cuda_check(ctx, cudaGetLastError(), "gaunt kernel")) || (rc = sync(ctx))) { hfx_destroy(ctx); return rc; }
    *out = ctx;
    return HFX_OK;
}

int hfx_set_radial(hfx_ctx *ctx, int atom, const double *R, const double *mu) {
    if (!ctx) return HFX_EINVAL;
    if (atom < 0 || atom >= ctx->sys.n_atoms || !R || !mu) return set_err(ctx, HFX_EINVAL, "set_radial: bad atom or pointer");
    int nLP = (ctx->sys.Lmax + 1) * ctx->P, nlp = ctx->nlp;
    size_t nR = (size_t)nLP * nlp * nlp;
    if (!finite_all(R, nR) || !finite_all(mu, nLP)) return set_err(ctx, HFX_ENONFINITE, "set_radial: non-finite value");
    double mx = 0.0;
    for (size_t i = 0; i < nR; ++i) mx = std::max(mx, std::fabs(R[i]));
    for (int t = 0; t < nLP; ++t)
        for (int i = 0; i < nlp; ++i)
            for (int j = 0; j < i; ++j)
                if (std::fabs(R[(size_t)t * nlp * nlp + i * nlp + j] - R[(size_t)t * nlp * nlp + j * nlp + i]) > 1e-12 * std::max(1.0, mx))
                    return set_err(ctx, HFX_EINVAL, "set_radial: R is not symmetric in (lp) <-> (l'p')");
    int rc = h2d(ctx, ctx->d_R + (size_t)atom * nR, R, nR);
    if (!rc) rc = h2d(ctx, ctx->d_mu + (size_t)atom * nLP, mu, nLP);
    if (!rc) rc = sync(ctx);
    if (rc) return rc;
    ctx->rset[atom] = 1;
    ctx->coulomb_dirty = true;
    ctx->built = false;
    return HFX_OK;
}

int hfx_set_kpoint(hfx_ctx *ctx, int ik, int n_bands, int n_occ, int npw, const int *G, const double *c,
                   const double *A) {
    if (!ctx) return HFX_EINVAL;
    if (ik < 0 || ik >= ctx->nk) return set_err(ctx, HFX_EINVAL, "set_kpoint: k index out of range");
    if (n_bands < 1 || n_bands > 4096 || n_occ < 0 || n_occ > n_bands || npw < 1 || npw > (1 << 20) || !G || !c || !A)
        return set_err(ctx, HFX_EINVAL, "set_kpoint: bad band counts, plane-wave count or pointer");
    for (int i = 0; i < 3 * npw; ++i)
        if (G[i] < -512 || G[i] > 512) return set_err(ctx, HFX_EINVAL, "set_kpoint: |G| component above 512");
    size_t nc = (size_t)n_bands * npw * 2, nA = (size_t)n_bands * ctx->sys.n_atoms * ctx->nlmp * 2;
    if (!finite_all(c, nc) || !finite_all(A, nA)) return set_err(ctx, HFX_ENONFINITE, "set_kpoint: non-finite coefficient");
    KPoint &k = ctx->kp[ik];
    if (k.set && (k.nb != n_bands || k.npw != npw)) {
        dfree(k.d_G); dfree(k.d_c); dfree(k.d_A);
        k.d_G = nullptr; k.d_c = nullptr; k.d_A = nullptr;
    }
    int rc = HFX_OK;
    if (!k.d_G && ((rc = dalloc(ctx, &k.d_G, (size_t)3 * npw)) || (rc = dalloc(ctx, &k.d_c, nc / 2)) ||
                   (rc = dalloc(ctx, &k.d_A, nA / 2))))
        return rc;
    if ((rc = h2d(ctx, k.d_G, G, (size_t)3 * npw)) || (rc = h2d(ctx, k.d_c, reinterpret_cast<const double2 *>(c), nc / 2)) ||
        (rc = h2d(ctx, k.d_A, reinterpret_cast<const double2 *>(A), nA / 2)))
        return rc;
    bool gchanged = !k.set || k.G.size() != (size_t)3 * npw || std::memcmp(k.G.data(), G, sizeof(int) * 3 * npw) != 0;
    if (gchanged || k.nb != n_bands || k.no != n_occ || k.npw != npw) ++ctx->struct_epoch;
    if (gchanged) k.G.assign(G, G + 3 * npw);
    k.nb = n_bands;
    k.no = n_occ;
    k.npw = npw;
    k.set = true;
    ctx->built = false;
    return HFX_OK;
}

int hfx_set_coulomb(hfx_ctx *ctx, int iq, int n_ipw, const int *G_aux, const double *v) {
    if (!ctx) return HFX_EINVAL;
    if (iq < 0 || iq >= ctx->nk) return set_err(ctx, HFX_EINVAL, "set_coulomb: q index out of range");
    if (n_ipw < 0 || n_ipw > (1 << 16) || (n_ipw > 0 && !G_aux) || !v) return set_err(ctx, HFX_EINVAL, "set_coulomb: bad size or pointer");
    for (int i = 0; i < 3 * n_ipw; ++i)
        if (G_aux[i] < -512 || G_aux[i] > 512) return set_err(ctx, HFX_EINVAL, "set_coulomb: |G| component above 512");
    int naux = ctx->nmt + n_ipw;
    size_t nv = (size_t)naux * naux * 2;
    if (!finite_all(v, nv)) return set_err(ctx, HFX_ENONFINITE, "set_coulomb: non-finite element");
    double mx = 0.0, dev = 0.0;
    for (size_t i = 0; i < nv; ++i) mx = std::max(mx, std::fabs(v[i]));
    for (int i = 0; i < naux; ++i)
        for (int j = 0; j <= i; ++j) {
            const double *a = v + 2 * ((size_t)i * naux + j), *b = v + 2 * ((size_t)j * naux + i);
            dev = std::max(dev, std::fabs(a[0] - b[0]) + std::fabs(a[1] + b[1]));
        }
    if (dev > ctx->opt.herm_tol * std::max(mx, 1e-300)) return set_err(ctx, HFX_ENOTHERM, "set_coulomb: v(q) is not Hermitian");
    QPoint &q = ctx->qp[iq];
    if (q.set && q.nipw != n_ipw) {
        dfree(q.d_G); dfree(q.d_v); dfree(q.d_VD); dfree(q.d_VB);
        q.d_G = nullptr; q.d_v = nullptr; q.d_VD = nullptr; q.d_VB = nullptr;
    }
    int rc = HFX_OK;
    if (!q.d_v && ((rc = dalloc(ctx, &q.d_G, (size_t)3 * std::max(n_ipw, 1))) || (rc = dalloc(ctx, &q.d_v, nv / 2))))
        return rc;
    if ((rc = h2d(ctx, q.d_G, G_aux, (size_t)3 * n_ipw)) || (rc = h2d(ctx, q.d_v, reinterpret_cast<const double2 *>(v), nv / 2)) ||
        (rc = sync(ctx)))
        return rc;
    if (!q.set || q.nipw != n_ipw || q.G.size() != (size_t)3 * n_ipw ||
        (n_ipw > 0 && std::memcmp(q.G.data(), G_aux, sizeof(int) * 3 * n_ipw) != 0))
        ++ctx->struct_epoch;
    q.G.assign(G_aux, G_aux + 3 * n_ipw);
    q.nipw = n_ipw;
    q.set = true;
    ctx->coulomb_dirty = true;
    ctx->built = false;
    return HFX_OK;
}

int hfx_set_products(hfx_ctx *ctx, int ik, int iq, const double *Z) {
    if (!ctx) return HFX_EINVAL;
    if (ik < 0 || ik >= ctx->nk || iq < 0 || iq >= ctx->nk) return set_err(ctx, HFX_EINVAL, "set_products: index out of range");
    auto key = std::make_pair(ik, iq);
    auto it = ctx->zover.find(key);
    if (!Z) {
        if (it != ctx->zover.end()) { dfree(it->second); ctx->zover.erase(it); }
        ctx->built = false;
        return HFX_OK;
    }
    const KPoint &k = ctx->kp[ik];
    const QPoint &q = ctx->qp[iq];
    if (!k.set || !q.set) return set_err(ctx, HFX_EMISSING, "set_products: set_kpoint(k) and set_coulomb(q) come first");
    int jk[3] = {ik / (ctx->sys.mesh[1] * ctx->sys.mesh[2]), (ik / ctx->sys.mesh[2]) % ctx->sys.mesh[1], ik % ctx->sys.mesh[2]};
    int jq[3] = {iq / (ctx->sys.mesh[1] * ctx->sys.mesh[2]), (iq / ctx->sys.mesh[2]) % ctx->sys.mesh[1], iq % ctx->sys.mesh[2]};
    int jp[3];
    for (int x = 0; x < 3; ++x) jp[x] = ((jk[x] - jq[x]) % ctx->sys.mesh[x] + ctx->sys.mesh[x]) % ctx->sys.mesh[x];
    int ikp = (jp[0] * ctx->sys.mesh[1] + jp[1]) * ctx->sys.mesh[2] + jp[2];
    if (!ctx->kp[ikp].set) return set_err(ctx, HFX_EMISSING, "set_products: set_kpoint(k - q) comes first");
    size_t n = (size_t)(ctx->nmt + q.nipw) * ctx->kp[ikp].no * k.nb;
    if (!finite_all(Z, 2 * n)) return set_err(ctx, HFX_ENONFINITE, "set_products: non-finite element");
    double2 *d = nullptr;
    int rc = HFX_OK;
    if (it != ctx->zover.end()) { dfree(it->second); ctx->zover.erase(it); }
    if ((rc = dalloc(ctx, &d, std::max<size_t>(n, 1)))) return rc;
    if ((rc = h2d(ctx, d, reinterpret_cast<const double2 *>(Z), n)) || (rc = sync(ctx))) { dfree(d); return rc; }
    ctx->zover[key] = d;
    ctx->built = false;
    return HFX_OK;
}

void hfx_destroy(hfx_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    for (auto &k : ctx->kp) { dfree(k.d_G); dfree(k.d_c); dfree(k.d_A); }
    for (auto &q : ctx->qp) { dfree(q.d_G); dfree(q.d_v); dfree(q.d_VD); dfree(q.d_VB); }
    for (auto &z : ctx->zover) dfree(z.second);
    for (auto &z : ctx->zkeep) dfree(z.second);
    for (auto *v : ctx->d_V) dfree(v);
    dfree(ctx->d_R); dfree(ctx->d_mu); dfree(ctx->d_T); dfree(ctx->d_gaunt); dfree(ctx->d_posf);
    dfree(ctx->d_err); dfree(ctx->d_Ex);
    Scratch *all[] = {&ctx->s_theta, &ctx->s_thpsi, &ctx->s_B,    &ctx->s_zc,   &ctx->s_zs,   &ctx->s_ys,
                      &ctx->s_y64,   &ctx->s_praw,  &ctx->s_vacc, &ctx->s_pairs, &ctx->s_qd,  &ctx->s_misc,
                      &ctx->s_ap,    &ctx->s_aexp,  &ctx->s_xexp, &ctx->s_zipw, &ctx->s_cgT, &ctx->s_cgZ};
    for (Scratch *s : all) dfree(s->p);
    delete ctx;
}

}  // extern "C"

// =====================================================================
// build
// =====================================================================
namespace {

struct Geometry {                 // integer boxes of the interstitial convolution
    int tlo[3], tdim[3];          // T_n(K) box: K = G + G1 - G0
    int dlo[3], ddim[3];          // Theta box: K - G2
};

Geometry boxes(hfx_ctx *ctx) {
    Geometry g;
    int amin[3], amax[3], pmin[3], pmax[3];
    for (int x = 0; x < 3; ++x) { amin[x] = pmin[x] = 1 << 29; amax[x] = pmax[x] = -(1 << 29); }
    for (auto &q : ctx->qp)
        for (size_t i = 0; i < q.G.size(); ++i) { int x = i % 3; amin[x] = std::min(amin[x], q.G[i]); amax[x] = std::max(amax[x], q.G[i]); }
    for (auto &k : ctx->kp)
        for (size_t i = 0; i < k.G.size(); ++i) { int x = i % 3; pmin[x] = std::min(pmin[x], k.G[i]); pmax[x] = std::max(pmax[x], k.G[i]); }
    for (int x = 0; x < 3; ++x) {
        if (amin[x] > amax[x]) { amin[x] = amax[x] = 0; }
        g.tlo[x] = amin[x] + pmin[x];          // -G0 in {0, 1}
        g.tdim[x] = (amax[x] + pmax[x] + 1) - g.tlo[x] + 1;
        g.dlo[x] = g.tlo[x] - pmax[x];
        g.ddim[x] = (g.tlo[x] + g.tdim[x] - 1 - pmin[x]) - g.dlo[x] + 1;
    }
    return g;
}

void fold(hfx_ctx *ctx, int ik, int iq, int *ikp, int *g0) {
    const int *M = ctx->sys.mesh;
    int jk[3] = {ik / (M[1] * M[2]), (ik / M[2]) % M[1], ik % M[2]};
    int jq[3] = {iq / (M[1] * M[2]), (iq / M[2]) % M[1], iq % M[2]};
    int jp[3];
    for (int x = 0; x < 3; ++x) {
        int d = jk[x] - jq[x];
        jp[x] = ((d % M[x]) + M[x]) % M[x];
        g0[x] = (d - jp[x]) / M[x];
    }
    *ikp = (jp[0] * M[1] + jp[1]) * M[2] + jp[2];
}

// Transform every v(q) (FP64), decide the sparse form, build the split embedding.
int prepare_coulomb(hfx_ctx *ctx) {
    if (!ctx->coulomb_dirty) return HFX_OK;
    const hfx_system &s = ctx->sys;
    int P = ctx->P, rc;
    launch_transform_T(ctx->d_mu, ctx->d_T, s.n_atoms, s.Lmax, P, ctx->stream);
    bool want_sparse = ctx->opt.sparse != HFX_SPARSE_OFF && P > 1;
    unsigned long long *d_mx = nullptr;
    if ((rc = dalloc(ctx, &d_mx, 2 * (size_t)ctx->nk))) return rc;
    cudaMemsetAsync(d_mx, 0, 2 * ctx->nk * sizeof(unsigned long long), ctx->stream);
    bool sparse = want_sparse;
    for (int pass = 0; pass < 2; ++pass) {
        int N0 = sparse ? ctx->nch * (P - 1) : 0;
        for (int iq = 0; iq < ctx->nk; ++iq) {
            QPoint &q = ctx->qp[iq];
            int naux = ctx->nmt + q.nipw, D = naux - N0;
            dfree(q.d_VD); dfree(q.d_VB);
            q.d_VD = nullptr; q.d_VB = nullptr;
            if ((rc = dalloc(ctx, &q.d_VD, (size_t)D * naux)) || (rc = dalloc(ctx, &q.d_VB, (size_t)std::max(1, ctx->nch * (P - 1) * P)))) {
                dfree(d_mx);
                return rc;
            }
            cudaMemsetAsync(q.d_VB, 0, sizeof(double2) * std::max(1, ctx->nch * (P - 1) * P), ctx->stream);
            launch_transform_v(q.d_v, q.d_VD, q.d_VB, ctx->d_T, s.n_atoms, s.Lmax, P, q.nipw, sparse ? 1 : 0,
                               d_mx + 2 * iq, d_mx + 2 * iq + 1, ctx->stream);
        }
        if ((rc = cuda_check(ctx, cudaGetLastError(), "transform kernel")) || (rc = sync(ctx))) { dfree(d_mx); return rc; }
        if (!sparse) break;
        std::vector<unsigned long long> h(2 * ctx->nk);
        cudaMemcpy(h.data(), d_mx, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
        bool ok = true;
        for (int iq = 0; iq < ctx->nk; ++iq) {
            double off, ab;
            std::memcpy(&off, &h[2 * iq], 8);
            std::memcpy(&ab, &h[2 * iq + 1], 8);
            if (off > ctx->opt.sparse_tol * ab) ok = false;
        }
        if (ok) break;
        if (ctx->opt.sparse == HFX_SPARSE_ON) { dfree(d_mx); return set_err(ctx, HFX_ENOTSPARSE, "v(q) is not block-sparse after the multipole transform"); }
        sparse = false;  // AUTO: fall back to the dense products
    }
    dfree(d_mx);
    ctx->sparse_used = sparse;
    ctx->N0 = sparse ? ctx->nch * (P - 1) : 0;
    if (ctx->opt.precision == HFX_PREC_SLICED) {
        int maxD = 0;
        for (auto &q : ctx->qp) maxD = std::max(maxD, ctx->nmt + q.nipw - ctx->N0);
        int N0pad = (int)rup(ctx->N0, 64), Dpad = (int)rup(maxD, 128);
        int RS = 2 * (N0pad + Dpad), MP = 2 * Dpad;
        size_t per = (size_t)4 * MP * RS;
        if ((rc = scratch_reserve(ctx, ctx->s_ap, per * ctx->nk * sizeof(__nv_bfloat16))) ||
            (rc = scratch_reserve(ctx, ctx->s_aexp, (size_t)MP * ctx->nk * sizeof(int))))
            return rc;
        __nv_bfloat16 *ap = reinterpret_cast<__nv_bfloat16 *>(ctx->s_ap.p);
        int *aexp = reinterpret_cast<int *>(ctx->s_aexp.p);
        for (int iq = 0; iq < ctx->nk; ++iq) {
            QPoint &q = ctx->qp[iq];
            int naux = ctx->nmt + q.nipw;
            launch_build_ap(q.d_VD, ap + per * iq, aexp + (size_t)MP * iq, naux - ctx->N0, naux, ctx->N0, N0pad, Dpad, RS,
                            ctx->stream);
        }
        if ((rc = cuda_check(ctx, cudaGetLastError(), "slice embedding")) || (rc = sync(ctx))) return rc;
    }
    ctx->coulomb_dirty = false;
    return HFX_OK;
}

int prepare_q0(hfx_ctx *ctx) {
    if (ctx->q0_valid) return HFX_OK;
    size_t n = q0_partial_count(ctx->sys.mesh, ctx->opt.beta, ctx->sys.lattice);
    double *d_part = nullptr, *d_out = nullptr;
    int rc;
    if ((rc = dalloc(ctx, &d_part, n)) || (rc = dalloc(ctx, &d_out, 1))) { dfree(d_part); return rc; }
    launch_q0_bracket_impl(d_out, d_part, ctx->sys.mesh, ctx->B, ctx->omega, ctx->opt.beta, ctx->sys.lattice, ctx->stream);
    rc = cuda_check(ctx, cudaGetLastError(), "q0 kernel");
    if (!rc) rc = sync(ctx);
    if (!rc) rc = cuda_check(ctx, cudaMemcpy(&ctx->q0_bracket, d_out, sizeof(double), cudaMemcpyDeviceToHost), "q0 copy");
    dfree(d_part);
    dfree(d_out);
    if (!rc) ctx->q0_valid = true;
    return rc;
}

template <typename T> T *as(Scratch &s, size_t off_bytes = 0) { return reinterpret_cast<T *>((char *)s.p + off_bytes); }

struct Events {
    std::vector<cudaEvent_t> ev;
    cudaEvent_t make(hfx_ctx *ctx) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, ctx->stream);
        ev.push_back(e);
        return e;
    }
    ~Events() {
        for (auto e : ev) cudaEventDestroy(e);
    }
};

template <typename R>
int build_impl(hfx_ctx *ctx, const std::vector<int> &kset, int keep, hfx_stats *st) {
    using V = typename C2<R>::T;
    const bool tc = (ctx->opt.precision == HFX_PREC_SLICED);
    const hfx_system &s = ctx->sys;
    const int nk = ctx->nk, P = ctx->P;
    int rc;
    Events evs;
    cudaEvent_t e_start = evs.make(ctx);

    if ((rc = prepare_coulomb(ctx)) || (rc = prepare_q0(ctx))) return rc;
    const int N0 = ctx->N0, sparse = ctx->sparse_used ? 1 : 0;
    const int nch = ctx->nch, nmt = ctx->nmt;
    int naux_max = 0, nb_max = 0, no_max = 0, npw_max = 0, maxD = 0;
    for (auto &q : ctx->qp) { naux_max = std::max(naux_max, nmt + q.nipw); maxD = std::max(maxD, nmt + q.nipw - N0); }
    for (auto &k : ctx->kp) { nb_max = std::max(nb_max, k.nb); no_max = std::max(no_max, k.no); npw_max = std::max(npw_max, k.npw); }
    const long long RSc = naux_max;
    const int N0pad = (int)rup(N0, 64), Dpad = (int)rup(maxD, 128), HS = N0pad + Dpad, RS = 2 * HS, MP = 2 * Dpad;

    // ---------------- per-k data: device pointer tables
    std::vector<const double2 *> hA(nk), hc(nk);
    std::vector<const int *> hG(nk), hGa(nk);
    std::vector<int> hnpw(nk), hnb(nk), hno(nk);
    for (int i = 0; i < nk; ++i) {
        hA[i] = ctx->kp[i].d_A; hc[i] = ctx->kp[i].d_c; hG[i] = ctx->kp[i].d_G; hGa[i] = ctx->qp[i].d_G;
        hnpw[i] = ctx->kp[i].npw; hnb[i] = ctx->kp[i].nb; hno[i] = ctx->kp[i].no;
    }
    Geometry geo = boxes(ctx);
    long long tbox = (long long)geo.tdim[0] * geo.tdim[1] * geo.tdim[2];
    long long dbox = (long long)geo.ddim[0] * geo.ddim[1] * geo.ddim[2];
    if (tbox > (1LL << 26) || dbox > (1LL << 27)) return set_err(ctx, HFX_EUNSUPPORTED, "plane-wave boxes too large");
    // which k carry the pairs: kset; which k' are needed: all (every k' = k - q)
    std::vector<char> need_k(nk, 0);
    for (int ik : kset) need_k[ik] = 1;

    // misc device tables: pointer arrays + per-k ints
    size_t off = 0;
    auto place = [&](size_t bytes) { size_t o = off; off = rup(off + bytes, 256); return o; };
    size_t o_A = place(nk * sizeof(void *)), o_c = place(nk * sizeof(void *)), o_G = place(nk * sizeof(void *)),
           o_Ga = place(nk * sizeof(void *)), o_npw = place(nk * sizeof(int)), o_nb = place(nk * sizeof(int)),
           o_no = place(nk * sizeof(int)), o_B = place(nk * sizeof(void *)), o_T = place(nk * sizeof(void *)),
           o_vacc = place(nk * sizeof(void *)), o_V = place(nk * sizeof(void *)), o_VB = place(nk * sizeof(void *));
    if ((rc = scratch_reserve(ctx, ctx->s_misc, off))) return rc;

    // per-k stage-1a and A4 outputs
    size_t bsz = (size_t)s.n_atoms * ctx->nLM * P * ctx->nlmp;
    std::vector<size_t> boff(nk), toff(nk);
    size_t btot = 0, ttot = 0;
    for (int i = 0; i < nk; ++i) { boff[i] = btot; btot += bsz * hnb[i]; toff[i] = ttot; ttot += (size_t)tbox * hnb[i]; }
    if ((rc = scratch_reserve(ctx, ctx->s_B, btot * sizeof(V))) || (rc = scratch_reserve(ctx, ctx->s_thpsi, ttot * sizeof(V))) ||
        (rc = scratch_reserve(ctx, ctx->s_theta, dbox * sizeof(double2))))
        return rc;
    std::vector<V *> hB(nk), hT(nk);
    for (int i = 0; i < nk; ++i) { hB[i] = as<V>(ctx->s_B) + boff[i]; hT[i] = as<V>(ctx->s_thpsi) + toff[i]; }
    // outputs
    size_t vtot = 0;
    std::vector<size_t> voff(nk);
    for (int i = 0; i < nk; ++i) { voff[i] = vtot; vtot += (size_t)hnb[i] * hnb[i]; }
    if ((rc = scratch_reserve(ctx, ctx->s_vacc, vtot * sizeof(double2)))) return rc;
    std::vector<double2 *> hvacc(nk), hV(nk);
    if (ctx->V_nb.size() != (size_t)nk) ctx->V_nb.assign(nk, 0);
    for (int i = 0; i < nk; ++i) {
        hvacc[i] = as<double2>(ctx->s_vacc) + voff[i];
        if (!ctx->d_V[i] || ctx->V_nb[i] != hnb[i]) {  // (re)allocate when the band window changed
            dfree(ctx->d_V[i]);
            ctx->d_V[i] = nullptr;
            if ((rc = dalloc(ctx, &ctx->d_V[i], (size_t)hnb[i] * hnb[i]))) return rc;
            ctx->V_nb[i] = hnb[i];
        }
        hV[i] = ctx->d_V[i];
    }
    char *misc = as<char>(ctx->s_misc);
    if ((rc = h2d(ctx, reinterpret_cast<const double2 **>(misc + o_A), hA.data(), nk)) ||
        (rc = h2d(ctx, reinterpret_cast<const double2 **>(misc + o_c), hc.data(), nk)) ||
        (rc = h2d(ctx, reinterpret_cast<const int **>(misc + o_G), hG.data(), nk)) ||
        (rc = h2d(ctx, reinterpret_cast<const int **>(misc + o_Ga), hGa.data(), nk)) ||
        (rc = h2d(ctx, reinterpret_cast<int *>(misc + o_npw), hnpw.data(), nk)) ||
        (rc = h2d(ctx, reinterpret_cast<int *>(misc + o_nb), hnb.data(), nk)) ||
        (rc = h2d(ctx, reinterpret_cast<int *>(misc + o_no), hno.data(), nk)) ||
        (rc = h2d(ctx, reinterpret_cast<V **>(misc + o_B), hB.data(), nk)) ||
        (rc = h2d(ctx, reinterpret_cast<V **>(misc + o_T), hT.data(), nk)) ||
        (rc = h2d(ctx, reinterpret_cast<double2 **>(misc + o_vacc), hvacc.data(), nk)) ||
        (rc = h2d(ctx, reinterpret_cast<double2 **>(misc + o_V), hV.data(), nk)))
        return rc;
    cudaMemsetAsync(ctx->s_vacc.p, 0, vtot * sizeof(double2), ctx->stream);

    // step function and the per-k precomputations (every k is some pair's k')
    launch_theta(as<double2>(ctx->s_theta), geo.dlo, geo.ddim, ctx->B, ctx->omega, ctx->d_posf, ctx->d_posf + 3 * s.n_atoms,
                 s.n_atoms, ctx->stream);
    for (int i = 0; i < nk; ++i) {
        if (!need_k[i]) continue;
        launch_bmat<R>(hA[i], ctx->d_R, ctx->d_T, ctx->d_gaunt, s.n_atoms, s.lmax, s.Lmax, P, hnb[i], sparse, hB[i], ctx->stream);
        if (!tc)
            launch_thetapsi<R>(as<double2>(ctx->s_theta), geo.dlo, geo.ddim, geo.tlo, geo.tdim, hc[i], hG[i], hnb[i],
                               hnpw[i], hT[i], ctx->stream);
    }
    if ((rc = cuda_check(ctx, cudaGetLastError(), "per-k kernels"))) return rc;
    ZmtTcState zmt_state;
    if (tc) {
        // T_n(K) and the operand slices of Z^MT on the tensor cores, once per build
        if ((rc = thetapsi_tc(ctx, kset, as<double2>(ctx->s_theta), geo.dlo, geo.ddim, geo.tlo, geo.tdim,
                              reinterpret_cast<double2 *>(ctx->s_thpsi.p), toff)))
            return rc;
        std::vector<double2 *> hB2(nk);
        for (int i = 0; i < nk; ++i) hB2[i] = reinterpret_cast<double2 *>(hB[i]);
        if ((rc = zmt_tc_prepare(ctx, zmt_state, kset, hB2, RSc, N0, sparse))) return rc;
    }

    // ---------------- q batches
    size_t budget = ctx->opt.work_bytes;
    if (!budget) {
        size_t fr = 0, totm = 0;
        cudaMemGetInfo(&fr, &totm);
        budget = (size_t)(0.55 * (double)fr);
    }
    // band block of the Z^H Y tiles: a multiple of 8 up to 64. A tile's MMA work and operand bytes grow
    // with NB (its 128-row A operand is padded), so pick the NB with the least nblk^2 * NB.
    int NB = 8;
    {
        long long best = 1LL << 60;
        for (int nbc = 8; nbc <= 64; nbc += 8) {
            long long nblk = (nb_max + nbc - 1) / nbc, cost = nblk * nblk * nbc;
            if (cost < best || (cost == best && nbc > NB)) { best = cost; NB = nbc; }
        }
    }
    auto qbytes = [&](int iq, long long *ncols_out, int *npairs_out) {
        long long nc = 0;
        int np = 0;
        size_t praw = 0;
        for (int ik : kset) {
            int ikp, g0[3];
            fold(ctx, ik, iq, &ikp, g0);
            nc += (long long)hno[ikp] * hnb[ik];
            ++np;
            if (tc) {
                int nblk = (hnb[ik] + NB - 1) / NB;
                praw += (size_t)nblk * nblk * (2 * NB) * (2 * NB) * sizeof(double);
            } else {
                praw += (size_t)hnb[ik] * hnb[ik] * sizeof(double2);
            }
        }
        *ncols_out = nc;
        *npairs_out = np;
        size_t b = (size_t)nc * RSc * sizeof(V) + praw + (size_t)nc * RSc * sizeof(double2);
        if (tc) b += (size_t)2 * 4 * nc * RS * sizeof(__nv_bfloat16) + 2 * nc * sizeof(int);
        return b;
    };
    std::vector<Batch> batches;
    {
        Batch cur;
        size_t used = 0;
        for (int iq = 0; iq < nk; ++iq) {
            long long nc;
            int np;
            size_t b = qbytes(iq, &nc, &np);
            if (!cur.qs.empty() && used + b > budget) { batches.push_back(cur); cur = Batch(); used = 0; }
            cur.qs.push_back(iq);
            used += b;
        }
        if (!cur.qs.empty()) batches.push_back(cur);
    }

    cudaEvent_t e_pre = evs.make(ctx);
    float ms_s1 = 0.f, ms_ct = 0.f;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> s1ev, ctev;
    double flops = 0.0, fl_apply = 0.0, fl_zhy = 0.0, fl_zipw = 0.0;
    int npairs_total = 0;
    // theta + per-k B (+ per-k Theta-psi in FP64; in the sliced build the Toeplitz
    // and band slices, the T product, and the two Z^MT operand slicings)
    int nlaunch = 1 + (tc ? (int)kset.size() + 5 : 2 * (int)kset.size());
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_zipw, ev_apply, ev_zhy, ev_zipw_gemm;

    for (Batch &bt : batches) {
        // columns and pairs
        long long col = 0;
        std::vector<int> kpair((size_t)nk * bt.qs.size(), -1);
        for (size_t qsl = 0; qsl < bt.qs.size(); ++qsl) {
            int iq = bt.qs[qsl];
            QDesc qd;
            qd.iq = iq;
            qd.nipw = ctx->qp[iq].nipw;
            qd.naux = nmt + qd.nipw;
            qd.D = qd.naux - N0;
            qd.colbase = col;
            qd.pair0 = (int)bt.pairs.size();
            for (int ik : kset) {
                PairDesc pr;
                pr.ik = ik;
                pr.iq = iq;
                fold(ctx, ik, iq, &pr.ikp, pr.g0);
                pr.nb = hnb[ik];
                pr.no = hno[pr.ikp];
                pr.col0 = col;
                pr.qslot = (int)qsl;
                pr.pad = 0;
                kpair[(size_t)ik * bt.qs.size() + qsl] = (int)bt.pairs.size();
                bt.pairs.push_back(pr);
                col += (long long)pr.no * pr.nb;
                // useful flops of the method (sparse form of Fig. 1 where used)
                double m = pr.no, n = pr.nb;
                double nnz = sparse ? (double)qd.D * qd.D + (double)nch * (P * P - 1) : (double)qd.naux * qd.naux;
                flops += 8.0 * m * n * (nnz + (double)qd.naux * n) + 8.0 * m * n * ctx->nlmp * nmt +
                         8.0 * m * n * qd.nipw * hnpw[pr.ikp];
                fl_apply += 8.0 * m * n * (double)qd.D * qd.D;
                fl_zhy += 8.0 * m * n * (double)qd.naux * n;
                fl_zipw += 8.0 * m * n * (double)qd.nipw * hnpw[pr.ikp];
            }
            qd.npairs = (int)bt.pairs.size() - qd.pair0;
            qd.ncols = col - qd.colbase;
            bt.qd.push_back(qd);
        }
        bt.ncols = col;
        int npairs = (int)bt.pairs.size();
        int nq = (int)bt.qs.size();
        npairs_total += npairs;
        long long maxcols = 0;
        for (auto &q : bt.qd) maxcols = std::max(maxcols, q.ncols);
        // praw offsets
        std::vector<long long> praw_off(npairs);
        long long praw_tot = 0;
        for (int i = 0; i < npairs; ++i) {
            praw_off[i] = praw_tot;
            if (tc) {
                int nblk = (bt.pairs[i].nb + NB - 1) / NB;
                praw_tot += (long long)nblk * nblk * (2 * NB) * (2 * NB);
            } else {
                praw_tot += 2LL * bt.pairs[i].nb * bt.pairs[i].nb;
            }
        }
        // per-k pair lists (ascending q) for the reduction
        std::vector<int> klist, kstart, klpairs;
        for (int ik : kset) {
            klist.push_back(ik);
            kstart.push_back((int)klpairs.size());
            for (int qsl = 0; qsl < nq; ++qsl) {
                int pi = kpair[(size_t)ik * nq + qsl];
                // a pair without occupied bands at k - q contributes nothing
                if (pi >= 0 && bt.pairs[pi].no > 0) klpairs.push_back(pi);
            }
        }
        kstart.push_back((int)klpairs.size());
        std::vector<const double2 *> hVB(nq), hVD(nq);
        for (int i = 0; i < nq; ++i) {
            hVB[i] = ctx->qp[bt.qs[i]].d_VB;
            hVD[i] = ctx->qp[bt.qs[i]].d_VD;
        }

        // device descriptors
        size_t o2 = 0;
        auto place2 = [&](size_t bytes) { size_t o = o2; o2 = rup(o2 + bytes, 256); return o; };
        size_t p_pairs = place2(npairs * sizeof(PairDesc)), p_qd = place2(nq * sizeof(QDesc)),
               p_kpair = place2(kpair.size() * sizeof(int)), p_praw = place2(npairs * sizeof(long long)),
               p_klist = place2(klist.size() * sizeof(int)), p_kstart = place2(kstart.size() * sizeof(int)),
               p_klp = place2(std::max<size_t>(1, klpairs.size()) * sizeof(int)), p_vb = place2(nq * sizeof(void *)),
               p_vd = place2(nq * sizeof(void *)),
               p_zg = place2(std::max(npairs, nq) * sizeof(ZGemmBatch)),
               p_tiles = place2((size_t)64 << 20);
        // per-batch tables of the tensor-core Z^MT product: offsets per (k, pair), phases, tiles
        const size_t zt_cap = tc ? rup((size_t)nk * (zmt_state.RB / 2) * 8, 256) + rup((size_t)nk * s.n_atoms * nk * 16, 256) +
                                       (size_t)nk * s.n_atoms * ((size_t)(nb_max * ctx->nLM * P + 127) / 128) *
                                           (size_t)(zmt_state.npairs_pad / 32 + 1) * 24 + 4096
                                 : 256;
        size_t p_zt = place2(zt_cap);
        if ((rc = scratch_reserve(ctx, ctx->s_pairs, o2))) return rc;
        char *dp = as<char>(ctx->s_pairs);
        PairDesc *d_pairs = reinterpret_cast<PairDesc *>(dp + p_pairs);
        QDesc *d_qd = reinterpret_cast<QDesc *>(dp + p_qd);
        int *d_kpair = reinterpret_cast<int *>(dp + p_kpair);
        long long *d_praw_off = reinterpret_cast<long long *>(dp + p_praw);
        if ((rc = h2d(ctx, d_pairs, bt.pairs.data(), npairs)) || (rc = h2d(ctx, d_qd, bt.qd.data(), nq)) ||
            (rc = h2d(ctx, d_kpair, kpair.data(), kpair.size())) || (rc = h2d(ctx, d_praw_off, praw_off.data(), npairs)) ||
            (rc = h2d(ctx, reinterpret_cast<int *>(dp + p_klist), klist.data(), klist.size())) ||
            (rc = h2d(ctx, reinterpret_cast<int *>(dp + p_kstart), kstart.data(), kstart.size())) ||
            (rc = h2d(ctx, reinterpret_cast<int *>(dp + p_klp), klpairs.data(), klpairs.size())) ||
            (rc = h2d(ctx, reinterpret_cast<const double2 **>(dp + p_vb), hVB.data(), nq)) ||
            (rc = h2d(ctx, reinterpret_cast<const double2 **>(dp + p_vd), hVD.data(), nq)))
            return rc;
        // working buffers
        if ((rc = scratch_reserve(ctx, ctx->s_zc, (size_t)bt.ncols * RSc * sizeof(V))) ||
            (rc = scratch_reserve(ctx, ctx->s_praw, (size_t)praw_tot * sizeof(double))))
            return rc;
        V *Zc = as<V>(ctx->s_zc);
        double *praw = as<double>(ctx->s_praw);

        cudaEvent_t e0 = evs.make(ctx);
        // ---- stage 1: projections
        if (tc) {
            if ((rc = zmt_tc_launch(ctx, zmt_state, bt.pairs, RSc, reinterpret_cast<double2 *>(Zc), dp + p_zt, zt_cap)))
                return rc;
        } else {
            launch_zmt<R>(d_pairs, npairs, d_qd, reinterpret_cast<V *const *>(misc + o_B),
                          reinterpret_cast<const double2 *const *>(misc + o_A), ctx->d_posf, s.mesh, s.n_atoms, ctx->nLM,
                          P, ctx->nlmp, N0, sparse, no_max, Zc, RSc, ctx->stream);
        }
        const int rowbase_ipw = nmt;  // N0 + n_ch = N_MT in the sparse order as well
        cudaEvent_t ez0 = evs.make(ctx);
        if (tc && sizeof(R) == 8) {
            ZipwTcInput zin;
            zin.kset = kset;
            zin.qs = bt.qs;
            zin.pairs = bt.pairs;
            zin.d_pairs = d_pairs;
            zin.d_ck = reinterpret_cast<const double2 *const *>(misc + o_c);
            zin.d_Gk = reinterpret_cast<const int *const *>(misc + o_G);
            zin.d_npw = reinterpret_cast<const int *>(misc + o_npw);
            zin.d_nb = reinterpret_cast<const int *>(misc + o_nb);
            zin.d_Tk = reinterpret_cast<const double2 *const *>(misc + o_T);
            zin.nb_max = nb_max;
            for (int x = 0; x < 3; ++x) { zin.tlo[x] = geo.tlo[x]; zin.tdim[x] = geo.tdim[x]; }
            zin.d_Z = reinterpret_cast<double2 *>(Zc);
            zin.RSc = RSc;
            cudaEventCreate(&zin.ev_gemm0);
            cudaEventCreate(&zin.ev_gemm1);
            evs.ev.push_back(zin.ev_gemm0);
            evs.ev.push_back(zin.ev_gemm1);
            if ((rc = zipw_tc_prepare_and_launch(ctx, zin))) return rc;
            ev_zipw_gemm.push_back({zin.ev_gemm0, zin.ev_gemm1});
        } else {
            rc = launch_zipw<R>(d_pairs, d_kpair, nk, nb_max, d_qd, nq, reinterpret_cast<V *const *>(misc + o_T), geo.tlo,
                                geo.tdim, reinterpret_cast<const double2 *const *>(misc + o_c),
                                reinterpret_cast<const int *const *>(misc + o_G), reinterpret_cast<const int *>(misc + o_npw),
                                npw_max, reinterpret_cast<const int *const *>(misc + o_Ga), reinterpret_cast<const int *>(misc + o_nb),
                                ctx->omega, rowbase_ipw, Zc, RSc, ctx->stream);
            if (rc) return set_err(ctx, rc, "interstitial kernel does not fit this size");
        }
        ev_zipw.push_back({ez0, evs.make(ctx)});
        nlaunch += tc ? 5 : 2;   // Z^MT; Z^IPW (sliced: C slices, T exponents, T slices, GEMM)
        for (int i = 0; i < npairs; ++i) {
            auto it = ctx->zover.find(std::make_pair(bt.pairs[i].ik, bt.pairs[i].iq));
            if (it == ctx->zover.end()) continue;
            launch_override<R>(it->second, bt.pairs[i], bt.qd[bt.pairs[i].qslot].naux, ctx->d_T, s.n_atoms, s.Lmax, P, N0,
                               sparse, Zc, RSc, nmt, ctx->stream);
            ++nlaunch;
        }
        if ((rc = cuda_check(ctx, cudaGetLastError(), "projection kernels"))) return rc;
        if (keep) {
            for (int i = 0; i < npairs; ++i) {
                const PairDesc &pr = bt.pairs[i];
                int naux = bt.qd[pr.qslot].naux;
                auto key = std::make_pair(pr.ik, pr.iq);
                auto it = ctx->zkeep.find(key);
                if (it != ctx->zkeep.end()) { dfree(it->second); ctx->zkeep.erase(it); }
                double2 *d = nullptr;
                if ((rc = dalloc(ctx, &d, (size_t)naux * pr.no * pr.nb))) return rc;
                ctx->zkeep[key] = d;
                launch_unpermute<R>(Zc, pr, naux, ctx->d_T, s.n_atoms, s.Lmax, P, N0, sparse, RSc, nmt, d, ctx->stream);
                ++nlaunch;
            }
        }
        cudaEvent_t e1 = evs.make(ctx);
        s1ev.push_back({e0, e1});

        // ---- contraction
        if (tc) {
            if ((rc = scratch_reserve(ctx, ctx->s_zs, (size_t)4 * bt.ncols * RS * sizeof(__nv_bfloat16))) ||
                (rc = scratch_reserve(ctx, ctx->s_ys, (size_t)4 * bt.ncols * RS * sizeof(__nv_bfloat16))) ||
                (rc = scratch_reserve(ctx, ctx->s_y64, (size_t)bt.ncols * RSc * sizeof(double2))) ||
                (rc = scratch_reserve(ctx, ctx->s_xexp, (size_t)2 * bt.ncols * sizeof(int))))
                return rc;
            __nv_bfloat16 *ZS = as<__nv_bfloat16>(ctx->s_zs), *YS = as<__nv_bfloat16>(ctx->s_ys);
            double2 *Yd = as<double2>(ctx->s_y64);
            int *zexp = as<int>(ctx->s_xexp), *yexp = zexp + bt.ncols;
            launch_slice_cols<V>(Zc, RSc, d_qd, nq, bt.ncols, maxcols, N0, N0pad, Dpad, RS, ZS, zexp, ctx->stream);
            if ((rc = cuda_check(ctx, cudaGetLastError(), "slice kernels"))) return rc;
            // the mu = 0 columns of the dense-block rows hold only each channel's
            // mu != 0 -> mu = 0 couplings: gemm1 leaves them out and the channel
            // block kernel, run after it, adds them
            const bool couple = sparse && std::is_same<V, double2>::value && block_y_couples(P, N0);
            cudaEvent_t ea0 = evs.make(ctx);
            if ((rc = launch_gemm1_tc(ctx, as<__nv_bfloat16>(ctx->s_ap), (long long)nk * 4 * MP, as<int>(ctx->s_aexp),
                                      bt.qd.data(), d_qd, nq, ZS, zexp, Yd, RSc, bt.ncols, N0, N0pad, Dpad, RS, couple,
                                      dp + p_tiles, (size_t)32 << 20)))
                return rc;
            cudaEvent_t ea1 = evs.make(ctx);
            launch_block_y<V>(d_qd, nq, reinterpret_cast<const double2 *const *>(dp + p_vb),
                              couple ? reinterpret_cast<const double2 *const *>(dp + p_vd) : nullptr, Zc, Yd, RSc, P, N0,
                              maxcols, ctx->stream);
            launch_slice_cols<double2>(Yd, RSc, d_qd, nq, bt.ncols, maxcols, N0, N0pad, Dpad, RS, YS, yexp, ctx->stream);
            cudaEvent_t ea2 = evs.make(ctx);
            if ((rc = launch_gemm2_tc(ctx, ZS, YS, zexp, yexp, bt.ncols, RS, HS, N0pad, bt.pairs.data(), d_pairs, npairs,
                                      d_qd, NB, d_praw_off, praw, dp + p_tiles + ((size_t)32 << 20), (size_t)32 << 20)))
                return rc;
            ev_apply.push_back({ea0, ea1});
            ev_zhy.push_back({ea2, evs.make(ctx)});
            nlaunch += 5;
        } else {
            if ((rc = scratch_reserve(ctx, ctx->s_y64, (size_t)bt.ncols * RSc * sizeof(double2)))) return rc;
            double2 *Y = as<double2>(ctx->s_y64);
            const double2 *Z64 = reinterpret_cast<const double2 *>(Zc);
            std::vector<ZGemmBatch> g1(nq);
            int maxM = 0, maxN = 0;
            for (int i = 0; i < nq; ++i) {
                const QDesc &q = bt.qd[i];
                ZGemmBatch &b = g1[i];
                b.A = ctx->qp[q.iq].d_VD;
                b.B = Z64 + q.colbase * RSc;
                b.C = Y + q.colbase * RSc + N0;
                b.M = q.D;
                b.N = (int)q.ncols;
                b.K1 = 1;
                b.K2 = q.naux;
                b.sAi = q.naux; b.sAk2 = 1; b.sAk1 = 0;
                b.sBk2 = 1; b.sBk1 = 0; b.sBj = RSc;
                b.sCi = 1; b.sCj = RSc;
                b.conjA = 0;
                maxM = std::max(maxM, b.M);
                maxN = std::max(maxN, b.N);
            }
            ZGemmBatch *d_zg = reinterpret_cast<ZGemmBatch *>(dp + p_zg);
            if ((rc = h2d(ctx, d_zg, g1.data(), nq))) return rc;
            cudaEvent_t ea0 = evs.make(ctx);
            launch_zgemm64(d_zg, nq, maxM, maxN, ctx->stream);
            ev_apply.push_back({ea0, evs.make(ctx)});
            launch_block64(d_qd, nq, reinterpret_cast<const double2 *const *>(dp + p_vb), Z64, Y, RSc, nch, P, N0, maxcols,
                           ctx->stream);
            if ((rc = cuda_check(ctx, cudaGetLastError(), "fp64 apply"))) return rc;
            // the Y rows of the dense block were written by the batched GEMM above;
            // wait for it before overwriting the descriptor table
            if ((rc = sync(ctx))) return rc;
            std::vector<ZGemmBatch> g2(npairs);
            int mx = 0;
            for (int i = 0; i < npairs; ++i) {
                const PairDesc &pr = bt.pairs[i];
                const QDesc &q = bt.qd[pr.qslot];
                ZGemmBatch &b = g2[i];
                b.A = Z64 + pr.col0 * RSc;
                b.B = Y + pr.col0 * RSc;
                b.C = reinterpret_cast<double2 *>(praw + praw_off[i]);
                b.M = pr.nb;
                b.N = pr.nb;
                b.K1 = pr.no;
                b.K2 = q.naux;
                b.sAi = RSc; b.sAk1 = (long long)pr.nb * RSc; b.sAk2 = 1;
                b.sBk1 = (long long)pr.nb * RSc; b.sBk2 = 1; b.sBj = RSc;
                b.sCi = pr.nb; b.sCj = 1;
                b.conjA = 1;
                mx = std::max(mx, pr.nb);
                if (pr.no == 0) { b.K1 = 1; b.K2 = 0; }
            }
            if ((rc = h2d(ctx, d_zg, g2.data(), npairs))) return rc;
            cudaEvent_t eh0 = evs.make(ctx);
            launch_zgemm64(d_zg, npairs, mx, mx, ctx->stream);
            ev_zhy.push_back({eh0, evs.make(ctx)});
            nlaunch += 3;
            if ((rc = cuda_check(ctx, cudaGetLastError(), "fp64 contraction"))) return rc;
        }
        launch_reduce_pairs(d_pairs, reinterpret_cast<int *>(dp + p_kstart), reinterpret_cast<int *>(dp + p_klp),
                            (int)klist.size(), reinterpret_cast<int *>(dp + p_klist), praw, d_praw_off, NB, tc ? 1 : 0,
                            reinterpret_cast<double2 *const *>(misc + o_vacc), reinterpret_cast<int *>(misc + o_nb), nb_max,
                            ctx->stream);
        if ((rc = cuda_check(ctx, cudaGetLastError(), "q reduction"))) return rc;
        ++nlaunch;
        cudaEvent_t e2 = evs.make(ctx);
        ctev.push_back({e1, e2});
        // descriptors are reused by the next batch
        if ((rc = sync(ctx))) return rc;
        if ((rc = check_dev_err(ctx))) return rc;
    }
    cudaEvent_t e_fin0 = evs.make(ctx);
    launch_finish(reinterpret_cast<double2 *const *>(misc + o_vacc), reinterpret_cast<double2 *const *>(misc + o_V),
                  reinterpret_cast<int *>(misc + o_nb), reinterpret_cast<int *>(misc + o_no), nk, nb_max, 1.0 / nk,
                  ctx->q0_bracket, ctx->opt.q0_term ? 1 : 0, ctx->d_Ex, ctx->stream);
    cudaEvent_t e_end = evs.make(ctx);
    if ((rc = cuda_check(ctx, cudaGetLastError(), "finish kernels")) || (rc = sync(ctx)) || (rc = check_dev_err(ctx))) return rc;
    if (st) {
        float t = 0.f;
        std::memset(st, 0, sizeof(*st));
        cudaEventElapsedTime(&t, e_start, e_end);
        st->ms_total = t;
        for (auto &pr : s1ev) { cudaEventElapsedTime(&t, pr.first, pr.second); ms_s1 += t; }
        for (auto &pr : ctev) { cudaEventElapsedTime(&t, pr.first, pr.second); ms_ct += t; }
        st->ms_stage1 = ms_s1;
        st->ms_contract = ms_ct;
        cudaEventElapsedTime(&t, e_fin0, e_end);
        st->ms_finish = t;
        st->useful_flops = flops;
        st->n_pairs = npairs_total;
        st->n_batches = (int)batches.size();
        st->sparse_used = ctx->sparse_used ? 1 : 0;
        st->n_launches = nlaunch + 2;
        auto sum = [&](std::vector<std::pair<cudaEvent_t, cudaEvent_t>> &v) {
            double tot = 0.0;
            for (auto &pr : v) { float x = 0.f; cudaEventElapsedTime(&x, pr.first, pr.second); tot += x; }
            return tot;
        };
        st->ms_zipw = ev_zipw_gemm.empty() ? sum(ev_zipw) : sum(ev_zipw_gemm);
        st->ms_apply = sum(ev_apply);
        st->ms_zhy = sum(ev_zhy);
        st->flops_apply = fl_apply;
        st->flops_zhy = fl_zhy;
        st->flops_zipw = fl_zipw;
    }
    (void)e_pre;
    ctx->built = true;
    return HFX_OK;
}

int check_ready(hfx_ctx *ctx) {
    for (int a = 0; a < ctx->sys.n_atoms; ++a)
        if (!ctx->rset[a]) return set_err(ctx, HFX_EMISSING, "set_radial missing for atom " + std::to_string(a));
    for (int i = 0; i < ctx->nk; ++i) {
        if (!ctx->kp[i].set) return set_err(ctx, HFX_EMISSING, "set_kpoint missing for k " + std::to_string(i));
        if (!ctx->qp[i].set) return set_err(ctx, HFX_EMISSING, "set_coulomb missing for q " + std::to_string(i));
    }
    return HFX_OK;
}

int build(hfx_ctx *ctx, const std::vector<int> &kset, int keep, hfx_stats *st) {
    int rc = check_ready(ctx);
    if (rc) return rc;
    rc = cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
    if (rc) return rc;
    return build_impl<double>(ctx, kset, keep, st);
}

}  // namespace

extern "C" {

int hfx_build_all(hfx_ctx *ctx, int keep_products, hfx_stats *st) {
    if (!ctx) return HFX_EINVAL;
    std::vector<int> all(ctx->nk);
    for (int i = 0; i < ctx->nk; ++i) all[i] = i;
    return build(ctx, all, keep_products, st);
}

int hfx_build_exchange(hfx_ctx *ctx, int ik, double *Vx, hfx_stats *st) {
    if (!ctx) return HFX_EINVAL;
    if (ik < 0 || ik >= ctx->nk || !Vx) return set_err(ctx, HFX_EINVAL, "build_exchange: bad k or pointer");
    int rc = build(ctx, std::vector<int>{ik}, 0, st);
    if (rc) return rc;
    ctx->built = false;  // only k was built
    int nb = ctx->kp[ik].nb;
    return cuda_check(ctx, cudaMemcpy(Vx, ctx->d_V[ik], sizeof(double2) * nb * nb, cudaMemcpyDeviceToHost), "copy V^x");
}

int hfx_get_exchange(hfx_ctx *ctx, int ik, double *Vx) {
    if (!ctx) return HFX_EINVAL;
    if (ik < 0 || ik >= ctx->nk || !Vx) return set_err(ctx, HFX_EINVAL, "get_exchange: bad k or pointer");
    if (!ctx->built) return set_err(ctx, HFX_EMISSING, "get_exchange: no complete build");
    int nb = ctx->kp[ik].nb;
    return cuda_check(ctx, cudaMemcpy(Vx, ctx->d_V[ik], sizeof(double2) * nb * nb, cudaMemcpyDeviceToHost), "copy V^x");
}

int hfx_exchange_device_ptr(hfx_ctx *ctx, int ik, const double **Vx_dev) {
    if (!ctx) return HFX_EINVAL;
    if (ik < 0 || ik >= ctx->nk || !Vx_dev) return set_err(ctx, HFX_EINVAL, "exchange_device_ptr: bad k or pointer");
    if (!ctx->built) return set_err(ctx, HFX_EMISSING, "exchange_device_ptr: no complete build");
    *Vx_dev = reinterpret_cast<const double *>(ctx->d_V[ik]);
    return HFX_OK;
}

int hfx_get_energy(hfx_ctx *ctx, double *Ex) {
    if (!ctx) return HFX_EINVAL;
    if (!Ex) return set_err(ctx, HFX_EINVAL, "get_energy: null pointer");
    if (!ctx->built) return set_err(ctx, HFX_EMISSING, "get_energy: no complete build");
    return cuda_check(ctx, cudaMemcpy(Ex, ctx->d_Ex, sizeof(double), cudaMemcpyDeviceToHost), "copy E_x");
}

int hfx_get_q0_bracket(hfx_ctx *ctx, double *b) {
    if (!ctx) return HFX_EINVAL;
    if (!b) return set_err(ctx, HFX_EINVAL, "get_q0_bracket: null pointer");
    int rc = prepare_q0(ctx);
    if (rc) return rc;
    *b = ctx->q0_bracket;
    return HFX_OK;
}

int hfx_get_products(hfx_ctx *ctx, int ik, int iq, double *Z) {
    if (!ctx) return HFX_EINVAL;
    if (ik < 0 || ik >= ctx->nk || iq < 0 || iq >= ctx->nk || !Z) return set_err(ctx, HFX_EINVAL, "get_products: bad index or pointer");
    auto it = ctx->zkeep.find(std::make_pair(ik, iq));
    if (it == ctx->zkeep.end()) return set_err(ctx, HFX_EMISSING, "get_products: build with keep_products first");
    int ikp, g0[3];
    fold(ctx, ik, iq, &ikp, g0);
    size_t n = (size_t)(ctx->nmt + ctx->qp[iq].nipw) * ctx->kp[ikp].no * ctx->kp[ik].nb;
    return cuda_check(ctx, cudaMemcpy(Z, it->second, n * sizeof(double2), cudaMemcpyDeviceToHost), "copy Z");
}

}  // extern "C"
