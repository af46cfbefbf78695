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

// Sec. III.D with the conventions of hfx_set_kpoint: phi(-r) = phi(r)^* holds
// when the plane-wave coefficients are real and, for every atom a with partner
// a' at -R_a + T_a, A^{a'}_{l,-m,p} = (-1)^(l+m) e^{i k.T_a} conj(A^a_{l,m,p}).
int check_inversion_bands(hfx_ctx *ctx, int ik, int nb, int npw, const double *c, const double *A) {
    const size_t nc = (size_t)nb * npw;
    double cmax = 0.0, cim = 0.0;
    for (size_t i = 0; i < nc; ++i) {
        cmax = std::max(cmax, std::max(std::fabs(c[2 * i]), std::fabs(c[2 * i + 1])));
        cim = std::max(cim, std::fabs(c[2 * i + 1]));
    }
    if (cim > ctx->opt.herm_tol * std::max(cmax, 1e-300))
        return set_err(ctx, HFX_EINVAL, "set_kpoint: plane-wave coefficients are not real (inversion mode)");
    const int *M = ctx->sys.mesh;
    const double kf[3] = {(double)(ik / (M[1] * M[2])) / M[0], (double)((ik / M[2]) % M[1]) / M[1], (double)(ik % M[2]) / M[2]};
    const int na = ctx->sys.n_atoms, nlmp = ctx->nlmp, lmax = ctx->sys.lmax;
    double amax = 0.0, dev = 0.0;
    for (size_t i = 0; i < (size_t)nb * na * nlmp * 2; ++i) amax = std::max(amax, std::fabs(A[i]));
    for (int a = 0; a < na; ++a) {
        const int b = ctx->partner[a];
        double kt = 0.0;   // k . T_a with T_a = R_a + R_a' (an integer vector in fractional units)
        for (int x = 0; x < 3; ++x) kt += kf[x] * std::floor(ctx->pos[3 * a + x] + ctx->pos[3 * b + x] + 0.5);
        kt *= 2.0 * M_PI;
        const double cr = std::cos(kt), ci = std::sin(kt);
        for (int n = 0; n < nb; ++n)
            for (int l = 0; l <= lmax; ++l)
                for (int m = -l; m <= l; ++m) {
                    const double sg = ((l + m) % 2 == 0) ? 1.0 : -1.0;
                    for (int p = 0; p < 2; ++p) {
                        const double *x = A + 2 * (((size_t)n * na + a) * nlmp + 2 * (l * l + l + m) + p);
                        const double *y = A + 2 * (((size_t)n * na + b) * nlmp + 2 * (l * l + l - m) + p);
                        // sg e^{i kt} conj(x)
                        const double er = sg * (cr * x[0] + ci * x[1]), ei = sg * (ci * x[0] - cr * x[1]);
                        dev = std::max(dev, std::fabs(y[0] - er) + std::fabs(y[1] - ei));
                    }
                }
    }
    if (dev > ctx->opt.herm_tol * std::max(amax, 1e-300))
        return set_err(ctx, HFX_EINVAL, "set_kpoint: MT coefficients do not satisfy phi(-r) = phi(r)^* (inversion mode)");
    return HFX_OK;
}

long long rup(long long x, long long m) { return (x + m - 1) / m * m; }

int sync(hfx_ctx *ctx) { return cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "stream synchronize"); }

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
    opt->use_graph = 1;
    opt->kp_term = 0;
    opt->kp_deg_tol = 1e-6;
    opt->tile_nb_zhy = 0;
    opt->tile_nb_zipw = 0;
    opt->test_fail_wait = 0;
    opt->inversion = 0;
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
    if ((opt.tile_nb_zhy && !gemm2_check_nb(opt.tile_nb_zhy)) || (opt.tile_nb_zipw && !zipw_tc_valid_nb(opt.tile_nb_zipw)))
        return HFX_EINVAL;
    if (!(opt.kp_deg_tol >= 0.0) || !std::isfinite(opt.kp_deg_tol)) return HFX_EINVAL;

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
    if (opt.inversion) {
        // Sec. III.D: every atom needs a partner at -R_a (up to a lattice vector)
        // with the same sphere radius
        ctx->partner.assign(sys->n_atoms, -1);
        for (int a = 0; a < sys->n_atoms; ++a) {
            for (int b = 0; b < sys->n_atoms && ctx->partner[a] < 0; ++b) {
                bool ok = std::fabs(sys->rmt[a] - sys->rmt[b]) < 1e-12;
                for (int x = 0; x < 3 && ok; ++x) {
                    const double d = sys->pos_frac[3 * a + x] + sys->pos_frac[3 * b + x];
                    ok = std::fabs(d - std::floor(d + 0.5)) < 1e-8;
                }
                if (ok) ctx->partner[a] = b;
            }
            if (ctx->partner[a] < 0) { delete ctx; return HFX_EINVAL; }
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
    ctx->hR.assign((size_t)sys->n_atoms * (sys->Lmax + 1) * ctx->P * ctx->nlp * ctx->nlp, 0.0);
    ctx->hmu.assign((size_t)sys->n_atoms * (sys->Lmax + 1) * ctx->P, 0.0);
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
        (rc = dalloc(ctx, &ctx->d_Tid, (size_t)sys->n_atoms * (sys->Lmax + 1) * ctx->P * ctx->P)) ||
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
    {
        const int P = ctx->P;
        std::vector<double> id((size_t)sys->n_atoms * (sys->Lmax + 1) * P * P, 0.0);
        for (size_t b = 0; b < (size_t)sys->n_atoms * (sys->Lmax + 1); ++b)
            for (int i = 0; i < P; ++i) id[b * P * P + (size_t)i * P + i] = 1.0;
        if ((rc = h2d(ctx, ctx->d_Tid, id.data(), id.size())) || (rc = sync(ctx))) { hfx_destroy(ctx); return rc; }
    }
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
    std::memcpy(ctx->hR.data() + (size_t)atom * nR, R, sizeof(double) * nR);
    std::memcpy(ctx->hmu.data() + (size_t)atom * nLP, mu, sizeof(double) * nLP);
    int rc = h2d(ctx, ctx->d_R + (size_t)atom * nR, R, nR);
    if (!rc) rc = h2d(ctx, ctx->d_mu + (size_t)atom * nLP, mu, nLP);
    if (!rc) rc = sync(ctx);
    if (rc) return rc;
    ctx->rset[atom] = 1;
    ctx->coulomb_dirty = true;
    ctx->T_valid = false;
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
    // inversion symmetry (Sec. III.D): phi(-r) = phi(r)^*, and two occupied bands
    // per complex column in the role m of k - q: X_j = X_{2j} - i X_{2j+1}
    const int nom = ctx->opt.inversion ? (n_occ + 1) / 2 : n_occ;
    const size_t nAb = (size_t)ctx->sys.n_atoms * ctx->nlmp;   // complex MT coefficients per band
    std::vector<double2> cm, Am;
    if (ctx->opt.inversion) {
        int rc0 = check_inversion_bands(ctx, ik, n_bands, npw, c, A);
        if (rc0) return rc0;
        cm.assign((size_t)nom * npw, make_double2(0.0, 0.0));
        Am.assign((size_t)nom * nAb, make_double2(0.0, 0.0));
        const double2 *c2 = reinterpret_cast<const double2 *>(c), *A2 = reinterpret_cast<const double2 *>(A);
        for (int j = 0; j < nom; ++j) {
            const bool two = 2 * j + 1 < n_occ;
            for (int g = 0; g < npw; ++g) {
                const double2 x = c2[(size_t)(2 * j) * npw + g], y = two ? c2[(size_t)(2 * j + 1) * npw + g] : make_double2(0.0, 0.0);
                cm[(size_t)j * npw + g] = make_double2(x.x + y.y, x.y - y.x);
            }
            for (size_t t = 0; t < nAb; ++t) {
                const double2 x = A2[(size_t)(2 * j) * nAb + t], y = two ? A2[(size_t)(2 * j + 1) * nAb + t] : make_double2(0.0, 0.0);
                Am[(size_t)j * nAb + t] = make_double2(x.x + y.y, x.y - y.x);
            }
        }
    }
    KPoint &k = ctx->kp[ik];
    auto drop_packed = [&]() {
        if (k.d_cm != k.d_c) dfree(k.d_cm);
        if (k.d_Am != k.d_A) dfree(k.d_Am);
        k.d_cm = nullptr; k.d_Am = nullptr;
    };
    if (k.set && (k.nb != n_bands || k.npw != npw)) {
        drop_packed();
        dfree(k.d_G); dfree(k.d_c); dfree(k.d_A);
        k.d_G = nullptr; k.d_c = nullptr; k.d_A = nullptr;
    }
    if (k.set && k.nom != nom) drop_packed();
    int rc = HFX_OK;
    if (!k.d_G && ((rc = dalloc(ctx, &k.d_G, (size_t)3 * npw)) || (rc = dalloc(ctx, &k.d_c, nc / 2)) ||
                   (rc = dalloc(ctx, &k.d_A, nA / 2))))
        return rc;
    if ((rc = h2d(ctx, k.d_G, G, (size_t)3 * npw)) || (rc = h2d(ctx, k.d_c, reinterpret_cast<const double2 *>(c), nc / 2)) ||
        (rc = h2d(ctx, k.d_A, reinterpret_cast<const double2 *>(A), nA / 2)))
        return rc;
    if (ctx->opt.inversion) {
        if (!k.d_cm && ((rc = dalloc(ctx, &k.d_cm, std::max<size_t>(1, (size_t)nom * npw))) ||
                        (rc = dalloc(ctx, &k.d_Am, std::max<size_t>(1, (size_t)nom * nAb)))))
            return rc;
        if ((rc = h2d(ctx, k.d_cm, cm.data(), cm.size())) || (rc = h2d(ctx, k.d_Am, Am.data(), Am.size())) ||
            (rc = sync(ctx)))
            return rc;
    } else {
        k.d_cm = k.d_c;
        k.d_Am = k.d_A;
    }
    bool gchanged = !k.set || k.G.size() != (size_t)3 * npw || std::memcmp(k.G.data(), G, sizeof(int) * 3 * npw) != 0;
    if (gchanged || k.nb != n_bands || k.no != n_occ || k.npw != npw) ++ctx->struct_epoch;
    if (gchanged) k.G.assign(G, G + 3 * npw);
    if (k.nb != n_bands) k.kp_set = false;   // the k.p inputs belong to the old band window
    if (k.nom != nom) ++ctx->struct_epoch;
    k.nb = n_bands;
    k.no = n_occ;
    k.nom = nom;
    k.npw = npw;
    k.set = true;
    ctx->built = false;
    return HFX_OK;
}

int hfx_set_coulomb(hfx_ctx *ctx, int iq, int n_ipw, const int *G_aux, const double *v, int ld, int layout) {
    if (!ctx) return HFX_EINVAL;
    if (iq < 0 || iq >= ctx->nk) return set_err(ctx, HFX_EINVAL, "set_coulomb: q index out of range");
    if (n_ipw < 0 || n_ipw > (1 << 16) || (n_ipw > 0 && !G_aux) || !v) return set_err(ctx, HFX_EINVAL, "set_coulomb: bad size or pointer");
    if (layout != HFX_LAYOUT_DENSE && layout != HFX_LAYOUT_TRANSFORMED && layout != HFX_LAYOUT_TRANSFORMED_ONSITE)
        return set_err(ctx, HFX_EINVAL, "set_coulomb: unknown layout");
    for (int i = 0; i < 3 * n_ipw; ++i)
        if (G_aux[i] < -512 || G_aux[i] > 512) return set_err(ctx, HFX_EINVAL, "set_coulomb: |G| component above 512");
    const int naux = ctx->nmt + n_ipw;
    if (ld < naux) return set_err(ctx, HFX_EINVAL, "set_coulomb: leading dimension below N_aux");
    const size_t nv = (size_t)naux * naux;
    // rows of stride ld into one contiguous N_aux x N_aux copy
    std::vector<double> vc;
    const double *vv = v;
    if (ld != naux) {
        vc.resize(2 * nv);
        for (int i = 0; i < naux; ++i) std::memcpy(vc.data() + 2 * (size_t)i * naux, v + 2 * (size_t)i * ld, 16 * (size_t)naux);
        vv = vc.data();
    }
    if (!finite_all(vv, 2 * nv)) return set_err(ctx, HFX_ENONFINITE, "set_coulomb: non-finite element");
    double mx = 0.0, dev = 0.0;
    for (size_t i = 0; i < 2 * nv; ++i) mx = std::max(mx, std::fabs(vv[i]));
    for (int i = 0; i < naux; ++i)
        for (int j = 0; j <= i; ++j) {
            const double *a = vv + 2 * ((size_t)i * naux + j), *b = vv + 2 * ((size_t)j * naux + i);
            dev = std::max(dev, std::fabs(a[0] - b[0]) + std::fabs(a[1] + b[1]));
        }
    if (dev > ctx->opt.herm_tol * std::max(mx, 1e-300)) return set_err(ctx, HFX_ENOTHERM, "set_coulomb: v(q) is not Hermitian");
    std::vector<double> vreal;
    if (ctx->opt.inversion) {
        // over the symmetrized MT functions of Sec. III.D, v(q) is real
        double im = 0.0;
        for (size_t i = 0; i < nv; ++i) im = std::max(im, std::fabs(vv[2 * i + 1]));
        if (im > ctx->opt.herm_tol * std::max(mx, 1e-300))
            return set_err(ctx, HFX_EINVAL, "set_coulomb: v(q) over the symmetrized basis is not real (inversion mode)");
        vreal.assign(vv, vv + 2 * nv);
        for (size_t i = 0; i < nv; ++i) vreal[2 * i + 1] = 0.0;
        vv = vreal.data();
    }
    QPoint &q = ctx->qp[iq];
    if (q.set && q.nipw != n_ipw) {
        dfree(q.d_G); dfree(q.d_v); dfree(q.d_VD); dfree(q.d_VB);
        q.d_G = nullptr; q.d_v = nullptr; q.d_VD = nullptr; q.d_VB = nullptr;
        q.vd_cap = q.vb_cap = 0;
    }
    int rc = HFX_OK;
    if (!q.d_v && ((rc = dalloc(ctx, &q.d_G, (size_t)3 * std::max(n_ipw, 1))) || (rc = dalloc(ctx, &q.d_v, nv))))
        return rc;
    if ((rc = h2d(ctx, q.d_G, G_aux, (size_t)3 * n_ipw)) || (rc = h2d(ctx, q.d_v, reinterpret_cast<const double2 *>(vv), nv)) ||
        (rc = sync(ctx)))
        return rc;
    if (!q.set || q.nipw != n_ipw || q.G.size() != (size_t)3 * n_ipw ||
        (n_ipw > 0 && std::memcmp(q.G.data(), G_aux, sizeof(int) * 3 * n_ipw) != 0))
        ++ctx->struct_epoch;
    q.G.assign(G_aux, G_aux + 3 * n_ipw);
    q.nipw = n_ipw;
    q.layout = layout;
    q.set = true;
    ctx->coulomb_dirty = true;
    ctx->built = false;
    return HFX_OK;
}

int hfx_set_momentum(hfx_ctx *ctx, int ik, const double *eps, const double *p) {
    if (!ctx) return HFX_EINVAL;
    if (ik < 0 || ik >= ctx->nk || !eps || !p) return set_err(ctx, HFX_EINVAL, "set_momentum: bad k or pointer");
    KPoint &k = ctx->kp[ik];
    if (!k.set) return set_err(ctx, HFX_EMISSING, "set_momentum: set_kpoint(k) comes first");
    const int nb = k.nb;
    const size_t np = (size_t)3 * nb * nb;
    if (!finite_all(eps, nb) || !finite_all(p, 2 * np)) return set_err(ctx, HFX_ENONFINITE, "set_momentum: non-finite value");
    double mx = 0.0, dev = 0.0;
    for (size_t i = 0; i < 2 * np; ++i) mx = std::max(mx, std::fabs(p[i]));
    for (int a = 0; a < 3; ++a)
        for (int m = 0; m < nb; ++m)
            for (int n = 0; n <= m; ++n) {
                const double *x = p + 2 * (((size_t)a * nb + m) * nb + n), *y = p + 2 * (((size_t)a * nb + n) * nb + m);
                dev = std::max(dev, std::fabs(x[0] + y[0]) + std::fabs(x[1] - y[1]));
            }
    if (dev > ctx->opt.herm_tol * std::max(mx, 1e-300))
        return set_err(ctx, HFX_EINVAL, "set_momentum: momentum elements are not anti-Hermitian");
    int rc = HFX_OK;
    if (k.kp_nb != nb) {
        dfree(k.d_eps); dfree(k.d_p); dfree(k.d_kp);
        k.d_eps = nullptr; k.d_p = nullptr; k.d_kp = nullptr;
        k.kp_nb = 0;
        if ((rc = dalloc(ctx, &k.d_eps, nb)) || (rc = dalloc(ctx, &k.d_p, np)) || (rc = dalloc(ctx, &k.d_kp, (size_t)nb * nb)))
            return rc;
        k.kp_nb = nb;
    }
    if ((rc = h2d(ctx, k.d_eps, eps, nb)) || (rc = h2d(ctx, k.d_p, reinterpret_cast<const double2 *>(p), np)) || (rc = sync(ctx)))
        return rc;
    k.kp_set = true;
    ctx->built = false;
    return HFX_OK;
}

int hfx_set_products(hfx_ctx *ctx, int ik, int iq, const double *Z) {
    if (!ctx) return HFX_EINVAL;
    if (ctx->opt.inversion) return set_err(ctx, HFX_EUNSUPPORTED, "set_products: not available with inversion symmetry");
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
    int ikp, g0[3];
    fold_kq(ctx, ik, iq, &ikp, g0);
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
    plan_release(ctx);
    for (auto &k : ctx->kp) {
        if (k.d_cm != k.d_c) dfree(k.d_cm);
        if (k.d_Am != k.d_A) dfree(k.d_Am);
        dfree(k.d_G); dfree(k.d_c); dfree(k.d_A); dfree(k.d_eps); dfree(k.d_p); dfree(k.d_kp);
    }
    for (auto &q : ctx->qp) { dfree(q.d_G); dfree(q.d_v); dfree(q.d_VD); dfree(q.d_VB); }
    for (auto &z : ctx->zover) dfree(z.second);
    for (auto &z : ctx->zkeep) dfree(z.second);
    for (auto *v : ctx->d_V) dfree(v);
    for (auto *v : ctx->d_S) dfree(v);
    dfree(ctx->s_lapw.p);
    dfree(ctx->s_lapw_tab.p);
    dfree(ctx->d_R); dfree(ctx->d_mu); dfree(ctx->d_T); dfree(ctx->d_Tid); dfree(ctx->d_gaunt); dfree(ctx->d_posf);
    dfree(ctx->d_err); dfree(ctx->d_Ex); dfree(ctx->d_radC);
    Scratch *all[] = {&ctx->s_theta, &ctx->s_thpsi, &ctx->s_B,    &ctx->s_zc,   &ctx->s_zs,   &ctx->s_ys,
                      &ctx->s_y64,   &ctx->s_praw,  &ctx->s_vacc, &ctx->s_pairs, &ctx->s_qd,  &ctx->s_misc,
                      &ctx->s_ap,    &ctx->s_aexp,  &ctx->s_xexp, &ctx->s_zipw, &ctx->s_cgT, &ctx->s_cgZ};
    for (Scratch *s : all) dfree(s->p);
    delete ctx;
}

}  // extern "C"

// =====================================================================
// once-per-SCF-cycle preparation (outside the build plan)
// =====================================================================
namespace {

// Multipole transforms T_aL from the current multipoles (Sec. III.C).
int prepare_T(hfx_ctx *ctx) {
    if (ctx->T_valid) return HFX_OK;
    launch_transform_T(ctx->d_mu, ctx->d_T, ctx->sys.n_atoms, ctx->sys.Lmax, ctx->P, ctx->stream);
    int rc = cuda_check(ctx, cudaGetLastError(), "transform kernel");
    if (!rc) ctx->T_valid = true;
    return rc;
}

// Transform every v(q) (FP64), decide the sparse form, build the split
// embedding.  The buffers of the transformed v(q) and of its slices keep their
// addresses across SCF cycles while the sizes stay (the build plan points at them).
int prepare_coulomb(hfx_ctx *ctx) {
    if (!ctx->coulomb_dirty) return HFX_OK;
    const hfx_system &s = ctx->sys;
    int P = ctx->P, rc;
    if ((rc = prepare_T(ctx))) return rc;
    bool onsite = false;
    for (auto &q : ctx->qp) onsite |= q.layout == HFX_LAYOUT_TRANSFORMED_ONSITE;
    if (onsite) {
        for (int a = 0; a < s.n_atoms; ++a)
            if (ctx->rad_set.size() != (size_t)s.n_atoms || !ctx->rad_set[a])
                return set_err(ctx, HFX_EMISSING, "TRANSFORMED_ONSITE: set_radial_functions missing for atom " + std::to_string(a));
        if (!ctx->d_radC && (rc = dalloc(ctx, &ctx->d_radC, ctx->rad_C.size()))) return rc;
        if ((rc = h2d(ctx, ctx->d_radC, ctx->rad_C.data(), ctx->rad_C.size()))) return rc;
        ctx->rad_C_dirty = false;
    }
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
            const size_t nvd = (size_t)D * naux, nvb = (size_t)std::max(1, ctx->nch * (P - 1) * P);
            if (q.vd_cap < nvd) {
                dfree(q.d_VD);
                q.d_VD = nullptr;
                q.vd_cap = 0;
                if ((rc = dalloc(ctx, &q.d_VD, nvd))) { dfree(d_mx); return rc; }
                q.vd_cap = nvd;
            }
            if (q.vb_cap < nvb) {
                dfree(q.d_VB);
                q.d_VB = nullptr;
                q.vb_cap = 0;
                if ((rc = dalloc(ctx, &q.d_VB, nvb))) { dfree(d_mx); return rc; }
                q.vb_cap = nvb;
            }
            cudaMemsetAsync(q.d_VB, 0, sizeof(double2) * nvb, ctx->stream);
            // the multipole-free rows and columns from the on-site blocks of the radial basis
            if (q.layout == HFX_LAYOUT_TRANSFORMED_ONSITE && pass == 0)
                launch_onsite_fill(q.d_v, naux, ctx->d_radC, ctx->d_T, s.n_atoms, s.Lmax, P, ctx->stream);
            // a v(q) given already transformed is only permuted (identity blocks)
            const double *T = q.layout != HFX_LAYOUT_DENSE ? ctx->d_Tid : ctx->d_T;
            launch_transform_v(q.d_v, q.d_VD, q.d_VB, T, s.n_atoms, s.Lmax, P, q.nipw, sparse ? 1 : 0, d_mx + 2 * iq,
                               d_mx + 2 * iq + 1, ctx->stream);
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
        cudaMemsetAsync(d_mx, 0, 2 * ctx->nk * sizeof(unsigned long long), ctx->stream);
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
            // the complex path interleaves the real and imaginary rows of U; the real
            // path (inversion symmetry) keeps them in two blocks
            launch_build_ap(q.d_VD, ap + per * iq, aexp + (size_t)MP * iq, naux - ctx->N0, naux, ctx->N0, N0pad, Dpad, RS,
                            ctx->opt.inversion ? 0 : 1, ctx->stream);
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

int check_ready(hfx_ctx *ctx) {
    for (int a = 0; a < ctx->sys.n_atoms; ++a)
        if (!ctx->rset[a]) return set_err(ctx, HFX_EMISSING, "set_radial missing for atom " + std::to_string(a));
    for (int i = 0; i < ctx->nk; ++i) {
        if (!ctx->kp[i].set) return set_err(ctx, HFX_EMISSING, "set_kpoint missing for k " + std::to_string(i));
        if (!ctx->qp[i].set) return set_err(ctx, HFX_EMISSING, "set_coulomb missing for q " + std::to_string(i));
    }
    if (ctx->opt.inversion) {
        // partner atoms are the same species: equal radial integrals and multipoles
        const size_t nR = ctx->hR.size() / ctx->sys.n_atoms, nmu = ctx->hmu.size() / ctx->sys.n_atoms;
        for (int a = 0; a < ctx->sys.n_atoms; ++a) {
            const int b = ctx->partner[a];
            double mx = 0.0, dev = 0.0;
            for (size_t i = 0; i < nR; ++i) {
                mx = std::max(mx, std::fabs(ctx->hR[a * nR + i]));
                dev = std::max(dev, std::fabs(ctx->hR[a * nR + i] - ctx->hR[b * nR + i]));
            }
            for (size_t i = 0; i < nmu; ++i) {
                mx = std::max(mx, std::fabs(ctx->hmu[a * nmu + i]));
                dev = std::max(dev, std::fabs(ctx->hmu[a * nmu + i] - ctx->hmu[b * nmu + i]));
            }
            if (dev > 1e-12 * std::max(mx, 1e-300))
                return set_err(ctx, HFX_EINVAL, "inversion: atoms " + std::to_string(a) + " and " + std::to_string(b) +
                                                    " differ in radial integrals or multipoles");
        }
    }
    return HFX_OK;
}

int build(hfx_ctx *ctx, const std::vector<int> &kset, int keep, hfx_stats *st) {
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (keep && ctx->opt.inversion)
        return set_err(ctx, HFX_EUNSUPPORTED, "keep_products: not available with inversion symmetry");
    if ((rc = cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice"))) return rc;
    if ((rc = prepare_coulomb(ctx)) || (rc = prepare_q0(ctx))) return rc;
    return build_run(ctx, kset, keep, st);
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

int hfx_get_transform(hfx_ctx *ctx, int atom, int L, double *T) {
    if (!ctx) return HFX_EINVAL;
    if (atom < 0 || atom >= ctx->sys.n_atoms || L < 0 || L > ctx->sys.Lmax || !T)
        return set_err(ctx, HFX_EINVAL, "get_transform: bad atom, L or pointer");
    if (!ctx->rset[atom]) return set_err(ctx, HFX_EMISSING, "get_transform: set_radial first");
    int rc = cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
    if (!rc) rc = prepare_T(ctx);
    if (!rc) rc = sync(ctx);
    if (rc) return rc;
    const int P = ctx->P;
    return cuda_check(ctx, cudaMemcpy(T, ctx->d_T + ((size_t)atom * (ctx->sys.Lmax + 1) + L) * P * P, sizeof(double) * P * P,
                                      cudaMemcpyDeviceToHost),
                      "copy T");
}

int hfx_get_products(hfx_ctx *ctx, int ik, int iq, double *Z) {
    if (!ctx) return HFX_EINVAL;
    if (ctx->opt.inversion) return set_err(ctx, HFX_EUNSUPPORTED, "get_products: not available with inversion symmetry");
    if (ik < 0 || ik >= ctx->nk || iq < 0 || iq >= ctx->nk || !Z) return set_err(ctx, HFX_EINVAL, "get_products: bad index or pointer");
    auto it = ctx->zkeep.find(std::make_pair(ik, iq));
    if (it == ctx->zkeep.end()) return set_err(ctx, HFX_EMISSING, "get_products: build with keep_products first");
    int ikp, g0[3];
    fold_kq(ctx, ik, iq, &ikp, g0);
    size_t n = (size_t)(ctx->nmt + ctx->qp[iq].nipw) * ctx->kp[ikp].no * ctx->kp[ik].nb;
    return cuda_check(ctx, cudaMemcpy(Z, it->second, n * sizeof(double2), cudaMemcpyDeviceToHost), "copy Z");
}

}  // extern "C"
