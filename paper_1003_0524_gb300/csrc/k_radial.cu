// k_radial.cu -- the muffin-tin side of the mixed product basis and of the
// Coulomb matrix, from the LAPW radial functions of an atom (Sec. III.B-C).
//
// For every L one thread block builds, in FP64:
//   - the products u_lp u_l'p' (lp <= l'p', |l - l'| <= L <= l + l'), each
//     normalised, and for L = 0 the constant function, projected out of them;
//   - the overlap matrix of the products and its eigenpairs (cyclic Jacobi);
//     eigenfunctions with eigenvalue above the threshold are linearly
//     independent, and the P largest of them (L = 0: P - 1 after the constant)
//     become the functions M_aLP, normalised, each with its largest eigenvector
//     component positive;
//   - the multipole moments mu_aLP = int M r^(L+2) dr (Sec. III.C), the radial
//     integrals R = int M u_lp u_l'p' r^2 dr, and the on-site Coulomb integrals
//     C_PP' = 4 pi/(2L+1) int int M_P(r) M_P'(r') r<^L/r>^(L+1) r^2 r'^2 dr dr'.
// A multipole-free combination of the M_aLP makes no potential outside its
// sphere, so every Coulomb matrix element with a mu = 0 function of the
// transform of Sec. III.C is one of these on-site integrals, the same for every
// q: launch_onsite_fill writes them into v_t (Fig. 1's channel blocks).
#include <cmath>
#include <string>
#include <vector>

#include "hfx_internal.cuh"

namespace hfx {

namespace {

constexpr int RB_THREADS = 256;
constexpr double kPi = 3.14159265358979323846;

__device__ double block_sum(double v, double *red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    const double t = red[0];
    __syncthreads();
    return t;
}

// One block per L.  Scratch per L: f [maxc][n_r], O and V [maxc][maxc].
__global__ void __launch_bounds__(RB_THREADS) mpb_radial_kernel(int n_r, const double *__restrict__ r,
                                                                const double *__restrict__ w, const double *__restrict__ u,
                                                                int lmax, int P, double thr, int maxc,
                                                                double *__restrict__ scr, double *__restrict__ M,
                                                                double *__restrict__ mu, double *__restrict__ R,
                                                                double *__restrict__ C, int *__restrict__ status) {
    const int L = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int nlp = 2 * (lmax + 1);
    double *f = scr + (size_t)L * ((size_t)maxc * n_r + 2 * (size_t)maxc * maxc);
    double *O = f + (size_t)maxc * n_r, *V = O + (size_t)maxc * maxc;
    extern __shared__ double sh[];
    double *red = sh;                  // [RB_THREADS]
    double *ev = red + RB_THREADS;     // [maxc]
    int *ia = reinterpret_cast<int *>(ev + maxc), *ib = ia + maxc;
    __shared__ int nc_s, fail, skip, pick[kMaxP];
    __shared__ double rot_c, rot_s, cst, scl[kMaxP];

    if (tid == 0) {
        int nc = 0;
        for (int a = 0; a < nlp; ++a)
            for (int b = a; b < nlp; ++b) {
                const int la = a / 2, lb = b / 2;
                if (abs(la - lb) > L || L > la + lb) continue;
                ia[nc] = a;
                ib[nc] = b;
                ++nc;
            }
        nc_s = nc;
        fail = 0;
    }
    __syncthreads();
    int nc = nc_s;
    for (size_t e = tid; e < (size_t)nc * n_r; e += nt) {
        const int c = (int)(e / n_r), i = (int)(e % n_r);
        f[e] = u[(size_t)ia[c] * n_r + i] * u[(size_t)ib[c] * n_r + i];
    }
    __syncthreads();
    // normalise; a product that vanishes identically is dropped
    for (int c = 0; c < nc; ++c) {
        double s = 0.0;
        for (int i = tid; i < n_r; i += nt) s += w[i] * r[i] * r[i] * f[(size_t)c * n_r + i] * f[(size_t)c * n_r + i];
        s = block_sum(s, red);
        if (s > 0.0) {
            const double inv = 1.0 / sqrt(s);
            for (int i = tid; i < n_r; i += nt) f[(size_t)c * n_r + i] *= inv;
        } else if (tid == 0) {
            ia[c] = -1;
        }
        __syncthreads();
    }
    if (tid == 0) {   // compact
        int k = 0;
        for (int c = 0; c < nc; ++c)
            if (ia[c] >= 0) {
                if (k != c)
                    for (int i = 0; i < n_r; ++i) f[(size_t)k * n_r + i] = f[(size_t)c * n_r + i];
                ia[k] = ia[c];
                ib[k] = ib[c];
                ++k;
            }
        nc_s = k;
    }
    __syncthreads();
    nc = nc_s;
    // L = 0: the constant function, projected out of the products
    if (L == 0) {
        double s = 0.0;
        for (int i = tid; i < n_r; i += nt) s += w[i] * r[i] * r[i];
        s = block_sum(s, red);
        if (tid == 0) cst = 1.0 / sqrt(s);
        __syncthreads();
        for (int c = 0; c < nc; ++c) {
            double d = 0.0;
            for (int i = tid; i < n_r; i += nt) d += w[i] * r[i] * r[i] * cst * f[(size_t)c * n_r + i];
            d = block_sum(d, red);
            for (int i = tid; i < n_r; i += nt) f[(size_t)c * n_r + i] -= d * cst;
            __syncthreads();
        }
    }
    // overlap matrix
    for (int e = tid; e < nc * nc; e += nt) {
        const int a = e / nc, b = e % nc;
        double o = 0.0;
        for (int i = 0; i < n_r; ++i) o += w[i] * r[i] * r[i] * f[(size_t)a * n_r + i] * f[(size_t)b * n_r + i];
        O[e] = o;
        V[e] = (a == b) ? 1.0 : 0.0;
    }
    __syncthreads();
    // cyclic Jacobi: at most 100 sweeps
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int e = tid; e < nc * nc; e += nt) {
            const double x = O[e] * O[e];
            tot += x;
            if (e / nc != e % nc) off += x;
        }
        off = block_sum(off, red);
        tot = block_sum(tot, red);
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < nc - 1; ++p)
            for (int q = p + 1; q < nc; ++q) {
                if (tid == 0) {
                    const double apq = O[p * nc + q];
                    skip = apq == 0.0;
                    if (!skip) {
                        const double theta = (O[q * nc + q] - O[p * nc + p]) / (2.0 * apq);
                        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        rot_c = 1.0 / sqrt(t * t + 1.0);
                        rot_s = t * rot_c;
                    }
                }
                __syncthreads();
                if (!skip) {
                    const double c = rot_c, sn = rot_s;
                    for (int k = tid; k < nc; k += nt) {
                        const double akp = O[k * nc + p], akq = O[k * nc + q];
                        O[k * nc + p] = c * akp - sn * akq;
                        O[k * nc + q] = sn * akp + c * akq;
                        const double vkp = V[k * nc + p], vkq = V[k * nc + q];
                        V[k * nc + p] = c * vkp - sn * vkq;
                        V[k * nc + q] = sn * vkp + c * vkq;
                    }
                    __syncthreads();
                    for (int k = tid; k < nc; k += nt) {
                        const double apk = O[p * nc + k], aqk = O[q * nc + k];
                        O[p * nc + k] = c * apk - sn * aqk;
                        O[q * nc + k] = sn * apk + c * aqk;
                    }
                }
                __syncthreads();
            }
    }
    for (int c = tid; c < nc; c += nt) ev[c] = O[c * nc + c];
    __syncthreads();
    // the largest eigenvalues above the threshold, descending; sign and scale
    const int want = (L == 0) ? P - 1 : P;
    if (tid == 0) {
        int got = 0;
        for (int k = 0; k < want; ++k) {
            int best = -1;
            for (int c = 0; c < nc; ++c) {
                bool used = false;
                for (int j = 0; j < got; ++j) used |= pick[j] == c;
                if (!used && ev[c] > thr && (best < 0 || ev[c] > ev[best])) best = c;
            }
            if (best < 0) break;
            pick[got++] = best;
        }
        if (got < want) {
            fail = 1;
            atomicMin(status, -(L + 1));
        } else {
            for (int k = 0; k < want; ++k) {
                const int e = pick[k];
                int big = 0;
                for (int c = 1; c < nc; ++c)
                    if (fabs(V[c * nc + e]) > fabs(V[big * nc + e])) big = c;
                scl[k] = (V[big * nc + e] >= 0 ? 1.0 : -1.0) / sqrt(ev[e]);
            }
        }
    }
    __syncthreads();
    if (fail) return;
    // the functions M_aLP on the grid
    double *ML = M + (size_t)L * P * n_r;
    for (size_t e = tid; e < (size_t)P * n_r; e += nt) {
        const int Pi = (int)(e / n_r), i = (int)(e % n_r);
        double v;
        if (L == 0 && Pi == 0) {
            v = cst;
        } else {
            const int k = (L == 0) ? Pi - 1 : Pi, ec = pick[k];
            double acc = 0.0;
            for (int c = 0; c < nc; ++c) acc += V[c * nc + ec] * f[(size_t)c * n_r + i];
            v = scl[k] * acc;
        }
        ML[e] = v;
    }
    __syncthreads();
    // multipole moments and radial integrals
    for (int e = tid; e < P * (1 + nlp * nlp); e += nt) {
        const int Pi = e / (1 + nlp * nlp), t = e % (1 + nlp * nlp);
        const double *m = ML + (size_t)Pi * n_r;
        double acc = 0.0;
        if (t == 0) {
            for (int i = 0; i < n_r; ++i) acc += w[i] * m[i] * pow(r[i], L + 2);
            mu[L * P + Pi] = acc;
        } else {
            const int a = (t - 1) / nlp, b = (t - 1) % nlp;
            for (int i = 0; i < n_r; ++i) acc += w[i] * r[i] * r[i] * m[i] * u[(size_t)a * n_r + i] * u[(size_t)b * n_r + i];
            R[(((size_t)L * P + Pi) * nlp + a) * nlp + b] = acc;
        }
    }
    // on-site Coulomb integrals (Laplace expansion, tensor-product quadrature)
    for (int Pi = 0; Pi < P; ++Pi)
        for (int Q = 0; Q < P; ++Q) {
            const double *m = ML + (size_t)Pi * n_r, *g = ML + (size_t)Q * n_r;
            double acc = 0.0;
            for (int i = tid; i < n_r; i += nt) {
                double inner = 0.0;
                for (int j = 0; j < n_r; ++j) {
                    const double rl = r[i] < r[j] ? r[i] : r[j], rg = r[i] < r[j] ? r[j] : r[i];
                    inner += w[j] * r[j] * r[j] * g[j] * pow(rl, L) / pow(rg, L + 1);
                }
                acc += w[i] * r[i] * r[i] * m[i] * inner;
            }
            acc = block_sum(acc, red);
            if (tid == 0) C[((size_t)L * P + Pi) * P + Q] = 4.0 * kPi / (2 * L + 1) * acc;
        }
}

// The mu = 0 rows and columns of v_t (transformed index positions, Sec. III.C):
// inside channel (a, L, M) the on-site block T C_aL T^T, zero elsewhere.
__global__ void onsite_fill_kernel(double2 *__restrict__ v, int naux, const double *__restrict__ C,
                                   const double *__restrict__ T, int n_atoms, int Lmax, int P) {
    const int nLM = (Lmax + 1) * (Lmax + 1);
    const long long nrow = (long long)n_atoms * nLM * (P - 1);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nrow * naux;
         e += (long long)gridDim.x * blockDim.x) {
        const long long rix = e / naux;
        const int J = (int)(e % naux);
        const int ch = (int)(rix / (P - 1)), i = 1 + (int)(rix % (P - 1));
        const int a = ch / nLM, L = (int)floor(sqrt((double)(ch % nLM)) + 1e-9);
        const int I = ch * P + i;
        double val = 0.0;
        if (J / P == ch && J < n_atoms * nLM * P) {
            const int j = J % P;
            const double *Ta = T + ((size_t)a * (Lmax + 1) + L) * P * P;
            const double *Ca = C + ((size_t)a * (Lmax + 1) + L) * P * P;
            for (int p = 0; p < P; ++p)
                for (int q = 0; q < P; ++q) val += Ta[i * P + p] * Ca[p * P + q] * Ta[j * P + q];
        }
        v[(size_t)I * naux + J] = make_double2(val, 0.0);
        v[(size_t)J * naux + I] = make_double2(val, 0.0);
    }
}

}  // namespace

void launch_onsite_fill(double2 *d_v, int naux, const double *d_C, const double *d_T, int n_atoms, int Lmax, int P,
                        cudaStream_t st) {
    if (P < 2) return;
    const long long n = (long long)n_atoms * (Lmax + 1) * (Lmax + 1) * (P - 1) * naux;
    long long g = (n + 255) / 256;
    if (g > 152LL * 32) g = 152LL * 32;
    onsite_fill_kernel<<<(unsigned)std::max<long long>(g, 1), 256, 0, st>>>(d_v, naux, d_C, d_T, n_atoms, Lmax, P);
}

}  // namespace hfx

using namespace hfx;

extern "C" {

int hfx_set_radial_functions(hfx_ctx *ctx, int atom, int n_r, const double *r, const double *w, const double *u,
                             double threshold) {
    if (!ctx) return HFX_EINVAL;
    const hfx_system &s = ctx->sys;
    if (atom < 0 || atom >= s.n_atoms || !r || !w || !u || n_r < 2 || n_r > 8192 || !(threshold > 0.0))
        return set_err(ctx, HFX_EINVAL, "set_radial_functions: bad atom, grid, pointer or threshold");
    if (ctx->P > kMaxP) return set_err(ctx, HFX_EUNSUPPORTED, "set_radial_functions: P above the kernel's limit");
    const int nlp = ctx->nlp, LP = (s.Lmax + 1) * ctx->P, P = ctx->P;
    for (int i = 0; i < n_r; ++i)
        if (!std::isfinite(r[i]) || !std::isfinite(w[i]) || r[i] <= 0.0 || r[i] > ctx->rmt[atom] * (1.0 + 1e-12) ||
            (i > 0 && r[i] <= r[i - 1]))
            return set_err(ctx, HFX_EINVAL, "set_radial_functions: grid must increase within (0, R_MT]");
    for (size_t i = 0; i < (size_t)nlp * n_r; ++i)
        if (!std::isfinite(u[i])) return set_err(ctx, HFX_ENONFINITE, "set_radial_functions: non-finite u");
    int rc = cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
    if (rc) return rc;
    const int maxc = nlp * (nlp + 1) / 2;
    const size_t per_L = (size_t)maxc * n_r + 2 * (size_t)maxc * maxc;
    double *d_in = nullptr, *d_scr = nullptr, *d_out = nullptr;
    int *d_status = nullptr;
    const size_t n_in = 2 * (size_t)n_r + (size_t)nlp * n_r;
    const size_t n_out = (size_t)LP * n_r + LP + (size_t)LP * nlp * nlp + (size_t)(s.Lmax + 1) * P * P;
    auto cleanup = [&]() { cudaFree(d_in); cudaFree(d_scr); cudaFree(d_out); cudaFree(d_status); };
    if ((rc = cuda_check(ctx, cudaMalloc(&d_in, n_in * sizeof(double)), "radial inputs")) ||
        (rc = cuda_check(ctx, cudaMalloc(&d_scr, per_L * (s.Lmax + 1) * sizeof(double)), "radial scratch")) ||
        (rc = cuda_check(ctx, cudaMalloc(&d_out, n_out * sizeof(double)), "radial outputs")) ||
        (rc = cuda_check(ctx, cudaMalloc(&d_status, sizeof(int)), "radial status"))) {
        cleanup();
        return rc;
    }
    std::vector<double> in(n_in);
    std::memcpy(in.data(), r, n_r * sizeof(double));
    std::memcpy(in.data() + n_r, w, n_r * sizeof(double));
    std::memcpy(in.data() + 2 * n_r, u, (size_t)nlp * n_r * sizeof(double));
    const int zero = 0;
    cudaMemcpyAsync(d_in, in.data(), n_in * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(d_status, &zero, sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
    double *dM = d_out, *dmu = dM + (size_t)LP * n_r, *dR = dmu + LP, *dC = dR + (size_t)LP * nlp * nlp;
    const size_t sm = (RB_THREADS + maxc) * sizeof(double) + 2 * (size_t)maxc * sizeof(int);
    mpb_radial_kernel<<<s.Lmax + 1, RB_THREADS, sm, ctx->stream>>>(n_r, d_in, d_in + n_r, d_in + 2 * n_r, s.lmax, P,
                                                                   threshold, maxc, d_scr, dM, dmu, dR, dC, d_status);
    std::vector<double> out(n_out);
    int status = 0;
    if ((rc = cuda_check(ctx, cudaGetLastError(), "radial kernel")) ||
        (rc = cuda_check(ctx, cudaMemcpyAsync(out.data(), d_out, n_out * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
                         "radial results")) ||
        (rc = cuda_check(ctx, cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
                         "radial status")) ||
        (rc = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "radial kernel"))) {
        cleanup();
        return rc;
    }
    cleanup();
    if (status < 0)
        return set_err(ctx, HFX_EINVAL, "set_radial_functions: fewer than P product functions above the threshold for L = " +
                                            std::to_string(-status - 1));
    // keep the basis; R and mu replace those of hfx_set_radial
    const double *M = out.data(), *mu = M + (size_t)LP * n_r, *R = mu + LP, *C = R + (size_t)LP * nlp * nlp;
    if (ctx->rad_M.size() != (size_t)s.n_atoms) {
        ctx->rad_M.assign(s.n_atoms, {});
        ctx->rad_nr.assign(s.n_atoms, 0);
        ctx->rad_C.assign((size_t)s.n_atoms * (s.Lmax + 1) * P * P, 0.0);
        ctx->rad_set.assign(s.n_atoms, 0);
    }
    ctx->rad_M[atom].assign(M, M + (size_t)LP * n_r);
    ctx->rad_nr[atom] = n_r;
    std::memcpy(ctx->rad_C.data() + (size_t)atom * (s.Lmax + 1) * P * P, C, sizeof(double) * (s.Lmax + 1) * P * P);
    ctx->rad_set[atom] = 1;
    ctx->rad_C_dirty = true;
    return hfx_set_radial(ctx, atom, R, mu);
}

int hfx_get_radial_basis(hfx_ctx *ctx, int atom, double *M, double *mu, double *R, double *C) {
    if (!ctx) return HFX_EINVAL;
    const hfx_system &s = ctx->sys;
    if (atom < 0 || atom >= s.n_atoms) return set_err(ctx, HFX_EINVAL, "get_radial_basis: bad atom");
    if (ctx->rad_set.size() != (size_t)s.n_atoms || !ctx->rad_set[atom])
        return set_err(ctx, HFX_EMISSING, "get_radial_basis: set_radial_functions first");
    const int P = ctx->P, LP = (s.Lmax + 1) * P, nlp = ctx->nlp;
    if (M) std::memcpy(M, ctx->rad_M[atom].data(), sizeof(double) * ctx->rad_M[atom].size());
    if (mu) std::memcpy(mu, ctx->hmu.data() + (size_t)atom * LP, sizeof(double) * LP);
    if (R) std::memcpy(R, ctx->hR.data() + (size_t)atom * LP * nlp * nlp, sizeof(double) * (size_t)LP * nlp * nlp);
    if (C) std::memcpy(C, ctx->rad_C.data() + (size_t)atom * (s.Lmax + 1) * P * P, sizeof(double) * (s.Lmax + 1) * P * P);
    return HFX_OK;
}

}  // extern "C"
